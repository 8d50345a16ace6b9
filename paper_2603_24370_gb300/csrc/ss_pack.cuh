// ss_pack.cuh -- a packed pair of FP32 values (F2) whose arithmetic compiles to the
// FP32x2 instructions (FADD2 / FMUL2 / FFMA2), so that one instruction advances two
// independent evaluations of the same formula.
//
// The flow passes evaluate the same stencils and force at two RK stage inputs of
// every site (stages 1-2 in pass 1, 3-4 in pass 2). Stored interleaved as (Y_a, Y_b)
// pairs in shared memory, both stages load with one 8-byte shared load and compute
// with one packed instruction, in a single walk: the force templates of ss_device.cuh
// are instantiated with R = F2.
//
// Products are kept as a pending pair (M2) until they meet an addition, so that
// a * b + c becomes one fused multiply-add as the compiler would form it in scalar
// code (the rounding of each packed lane then matches a contracted scalar evaluation
// up to where the contraction is placed).
#pragma once
#include <cuda_runtime.h>

namespace ss {

struct F2 {
  float2 v;
  F2() = default;
  __device__ __forceinline__ F2(float2 a) : v(a) {}
  __device__ __forceinline__ F2(float s) : v(make_float2(s, s)) {}
  __device__ __forceinline__ F2(double s) : v(make_float2((float)s, (float)s)) {}
  __device__ __forceinline__ F2(int s) : v(make_float2((float)s, (float)s)) {}
  __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
};

// a pending product a * b
struct M2 {
  float2 a, b;
  __device__ __forceinline__ operator F2() const { return F2(__fmul2_rn(a, b)); }
};

__device__ __forceinline__ float2 neg2(float2 x) { return make_float2(-x.x, -x.y); }

__device__ __forceinline__ M2 operator*(F2 x, F2 y) { return M2{x.v, y.v}; }
__device__ __forceinline__ M2 operator*(M2 p, F2 y) { return M2{__fmul2_rn(p.a, p.b), y.v}; }
__device__ __forceinline__ M2 operator*(F2 x, M2 p) { return M2{x.v, __fmul2_rn(p.a, p.b)}; }
__device__ __forceinline__ M2 operator*(M2 p, M2 q) { return M2{__fmul2_rn(p.a, p.b), __fmul2_rn(q.a, q.b)}; }

__device__ __forceinline__ F2 operator-(F2 x) { return F2(neg2(x.v)); }
__device__ __forceinline__ M2 operator-(M2 p) { return M2{neg2(p.a), p.b}; }

__device__ __forceinline__ F2 operator+(F2 x, F2 y) { return F2(__fadd2_rn(x.v, y.v)); }
__device__ __forceinline__ F2 operator-(F2 x, F2 y) { return F2(__fadd2_rn(x.v, neg2(y.v))); }
__device__ __forceinline__ F2 operator+(M2 p, F2 y) { return F2(__ffma2_rn(p.a, p.b, y.v)); }
__device__ __forceinline__ F2 operator+(F2 x, M2 p) { return F2(__ffma2_rn(p.a, p.b, x.v)); }
__device__ __forceinline__ F2 operator-(M2 p, F2 y) { return F2(__ffma2_rn(p.a, p.b, neg2(y.v))); }
__device__ __forceinline__ F2 operator-(F2 x, M2 p) { return F2(__ffma2_rn(neg2(p.a), p.b, x.v)); }
__device__ __forceinline__ F2 operator+(M2 p, M2 q) { return F2(__ffma2_rn(p.a, p.b, __fmul2_rn(q.a, q.b))); }
__device__ __forceinline__ F2 operator-(M2 p, M2 q) { return F2(__ffma2_rn(p.a, p.b, neg2(__fmul2_rn(q.a, q.b)))); }

__device__ __forceinline__ F2& operator+=(F2& x, F2 y) { return x = x + y; }
__device__ __forceinline__ F2& operator-=(F2& x, F2 y) { return x = x - y; }
__device__ __forceinline__ F2& operator+=(F2& x, M2 p) { return x = x + p; }
__device__ __forceinline__ F2& operator-=(F2& x, M2 p) { return x = x - p; }
__device__ __forceinline__ F2& operator*=(F2& x, F2 y) { return x = F2(x * y); }

}  // namespace ss
