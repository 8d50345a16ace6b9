// ss_noalloc.cu -- ss_observables_noalloc: the observables reduction for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code whose device memory is owned by a
// framework's caching allocator or a fixed arena that must account for every byte,
// code running where an allocation would implicitly synchronize the device or could
// fail (a latency-critical loop, a process whose device memory is already fully
// reserved). For them this entry point evaluates the same observables as
// ss_observables on a caller-owned device field, with the same kernels, but keeps
// all of its scratch (the reduction's per-block partials, its arrival counter and
// the result record) in one file-scope device array of fixed size. It allocates
// nothing, neither through CUDA nor through any library.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>

#include "soliton.h"
#include "ss_internal.h"

using namespace ss;

namespace {

// At most this many thread blocks take part in the reduction (the kernel strides
// over tiles, so any grid size fits). 2048 partials of 64 B plus the record: 128.25 KB.
constexpr int NOALLOC_MAX_BLOCKS = 2048;
constexpr size_t NOALLOC_RECORD_BYTES = (sizeof(DevState) + 255) & ~size_t(255);
constexpr size_t NOALLOC_BYTES = NOALLOC_RECORD_BYTES + sizeof(ObsPartial) * NOALLOC_MAX_BLOCKS;

}  // namespace

// The scratch. Every GPU that loads the library holds it until the process exits;
// all calls on a device share it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {

// Copy the result record into the caller's output (grad_max = dx dy * max|G|).
__global__ void k_noalloc_out(const DevState* st, double area, double* out) {
  out[0] = st->obs_energy;
  out[1] = st->obs_charge;
  out[2] = st->obs_flux;
  out[3] = area * st->obs_gmax_raw;
  out[4] = st->obs_gmax_raw;
  out[5] = st->obs_normdev;
}

// The message is reported by ss_last_error() like every other call's.
int noalloc_fail(int code, const std::string& msg) {
  set_last_error(msg);
  return code;
}

}  // namespace

extern "C" int ss_observables_noalloc(int theory, const double* params, int n_params, const void* fields, int nx,
                                      int ny, double dx, double dy, int precision, double* out, void* cuda_stream) {
  if (!fields || !out) return noalloc_fail(SS_ERR_ARG, "ss_observables_noalloc: fields and out must be device pointers");
  if (nx < 5 || ny < 5) return noalloc_fail(SS_ERR_ARG, "ss_observables_noalloc: nx and ny must be >= 5");
  if (nx > 65536 || ny > 65536 || (long long)nx * ny > (1LL << 31))
    return noalloc_fail(SS_ERR_ARG,
                        "ss_observables_noalloc: grid larger than the supported maximum (nx, ny <= 65536, nx*ny <= 2^31)");
  if (!(dx > 0.0) || !(dy > 0.0) || !std::isfinite(dx) || !std::isfinite(dy))
    return noalloc_fail(SS_ERR_ARG, "ss_observables_noalloc: dx and dy must be positive and finite");
  if (precision != SS_FP32 && precision != SS_FP64 && precision != SS_FP32_PLAIN)
    return noalloc_fail(SS_ERR_ARG, "ss_observables_noalloc: precision must be SS_FP32, SS_FP32_PLAIN or SS_FP64");

  // couplings, validated and packed by the same routine as ss_set_theory's
  double k[NCOUP];
  int C = 0;
  const int rc = pack_couplings(theory, params, n_params, k, &C);
  if (rc != SS_OK) return rc;
  if (theory == SS_CHIRAL_MAGNET && k[10] > 0.0)
    return noalloc_fail(SS_ERR_ARG, "ss_observables_noalloc: demagnetisation needs a context (a Poisson solve)");
  if (theory == SS_BEC && k[4] > 0.0)
    return noalloc_fail(SS_ERR_ARG, "ss_observables_noalloc: a fixed atom number needs a context (its multiplier)");

  // set-up, on every call, with the caller's device current: the device address of
  // the scratch (the array's name is only a host-side stand-in). Looking it up each
  // time keeps no address that a device reset could leave stale.
  void* base = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
  if (e != cudaSuccess)
    return noalloc_fail(SS_ERR_CUDA, std::string("ss_observables_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));

  LaunchCtx L{};
  L.theory = theory == SS_ABELIAN_HIGGS ? TH_AH
             : theory == SS_CHIRAL_MAGNET ? TH_CM
             : theory == SS_BABY_SKYRME   ? TH_BS
             : theory == SS_SID           ? TH_SID
                                          : TH_BEC;
  L.prec = precision;
  L.nx = nx;
  L.ny = ny;
  L.plane = (size_t)nx * ny;
  L.dx = dx;
  L.dy = dy;
  std::memcpy(L.coup, k, sizeof(k));
  L.phi[0] = const_cast<void*>(fields);
  L.st = reinterpret_cast<DevState*>(base);
  L.opart = reinterpret_cast<ObsPartial*>(static_cast<char*>(base) + NOALLOC_RECORD_BYTES);
  L.ntiles_x = (nx + TX - 1) / TX;
  L.ntiles_y = (ny + TY - 1) / TY;
  const int g = obs_grid(L.theory, precision, L.ntiles_x * L.ntiles_y);
  L.obs_blocks = g < NOALLOC_MAX_BLOCKS ? g : NOALLOC_MAX_BLOCKS;

  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // the arrival counter must start at zero; the rest of the record is overwritten
  e = cudaMemsetAsync(&L.st->obs_ticket, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) e = launch_observables(L, 0, s);
  if (e == cudaSuccess) {
    k_noalloc_out<<<1, 1, 0, s>>>(L.st, dx * dy, out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return noalloc_fail(SS_ERR_CUDA, std::string("ss_observables_noalloc: ") + cudaGetErrorString(e));
  return SS_OK;
}
