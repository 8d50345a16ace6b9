// Host-only check of the kernels' per-site arithmetic (compiled by nvcc, run on the
// CPU): the cancellation-free energy differences used by the arrest test must equal
// e(a) - e(a - delta) of the same density functions evaluated in higher precision.
// Prints one line per case: "<name> <max relative error>".
#include <cmath>
#include <cstdio>
#include <cstdint>

#include "../../paper_2603_24370_gb300/csrc/ss_device.cuh"

using namespace ss;

static uint64_t rng_state = 0x1234abcdULL;
static double uni(double lo, double hi) {  // SplitMix64 draws
  rng_state += 0x9E3779B97F4A7C15ULL;
  uint64_t z = rng_state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return lo + (hi - lo) * ((z >> 11) * (1.0 / 9007199254740992.0));
}

template <typename R, typename H>
static void coup(int theory, Couplings<R>& k, Couplings<H>& kh) {
  double c[10] = {0};
  if (theory == TH_AH) { c[0] = 1.3; c[1] = 1.0; }
  else { c[0] = 1.0; c[1] = 0.9; c[2] = 0.15; c[3] = 0.6; c[5] = 1.0; c[7] = -1.0; }
  for (int i = 0; i < 10; ++i) { k.c[i] = (R)c[i]; kh.c[i] = (H)c[i]; }
}

// R: working type of the kernel, H: reference type
template <typename R, typename H>
static double check(int theory, double dscale) {
  const int C = theory == TH_AH ? 4 : 3;
  Couplings<R> k; Couplings<H> kh;
  coup(theory, k, kh);
  double worst = 0.0;
  for (int t = 0; t < 20000; ++t) {
    R a[4], ax[4], ay[4], d[4], dx[4], dy[4];
    for (int c = 0; c < C; ++c) {
      a[c] = (R)uni(-1, 1); ax[c] = (R)uni(-2, 2); ay[c] = (R)uni(-2, 2);
      d[c] = (R)(dscale * uni(-1, 1)); dx[c] = (R)(dscale * uni(-3, 3)); dy[c] = (R)(dscale * uni(-3, 3));
    }
    H A[4], AX[4], AY[4], B[4], BX[4], BY[4];
    for (int c = 0; c < C; ++c) {
      A[c] = a[c]; AX[c] = ax[c]; AY[c] = ay[c];
      B[c] = (H)a[c] - (H)d[c]; BX[c] = (H)ax[c] - (H)dx[c]; BY[c] = (H)ay[c] - (H)dy[c];
    }
    H ref, scale;
    R got;
    if (theory == TH_AH) {
      ref = density_ah<H>(kh, A, AX, AY) - density_ah<H>(kh, B, BX, BY);
      got = delta_density_ah<R>(k, a, ax, ay, d, dx, dy);
    } else {
      ref = density_cm<H>(kh, A, AX, AY) - density_cm<H>(kh, B, BX, BY);
      got = delta_density_cm<R>(k, a, ax, ay, d, dx, dy);
    }
    scale = std::fabs((double)ref) + 1e-300;
    const double err = std::fabs((double)got - (double)ref) / scale;
    if (err > worst) worst = err;
  }
  return worst;
}

int main() {
  for (double ds : {1e-1, 1e-3, 1e-6}) {
    std::printf("ah_f32_%g %.3e\n", ds, check<float, long double>(TH_AH, ds));
    std::printf("cm_f32_%g %.3e\n", ds, check<float, long double>(TH_CM, ds));
    std::printf("ah_f64_%g %.3e\n", ds, check<double, long double>(TH_AH, ds));
    std::printf("cm_f64_%g %.3e\n", ds, check<double, long double>(TH_CM, ds));
  }
  return 0;
}
