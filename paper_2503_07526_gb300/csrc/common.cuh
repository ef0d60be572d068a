// Internal helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "otf_md.h"

namespace otf {

// Per-thread error message behind md_last_error().
void set_error(const char *fmt, ...);
void clear_error();

// Device-side error bits, OR-ed into a status word by kernels and turned
// into MD_ESTATE by the host.
enum : unsigned {
  ERR_NONFINITE = 1u,      // a coordinate or velocity became NaN / Inf
  ERR_NBR_OVERFLOW = 2u,   // an atom has more neighbours than the list holds
  ERR_BAD_TYPE = 4u,       // an atom type outside [0, ntypes)
  ERR_PUSH_BACKLOG = 8u,   // more velocity pushes waiting than one blocked pass applies
  ERR_WINDOW = 16u,        // a tile's shared-memory window outgrew its capacity (MD_PAIR_TILES)
};

#define OTF_CUDA(call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      otf::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,      \
                     __LINE__);                                                              \
      return e_ == cudaErrorMemoryAllocation ? MD_ENOMEM : MD_ECUDA;                         \
    }                                                                                        \
  } while (0)

#define OTF_LAUNCH_CHECK()                                                                   \
  do {                                                                                       \
    cudaError_t e_ = cudaGetLastError();                                                     \
    if (e_ != cudaSuccess) {                                                                 \
      otf::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_), __FILE__,  \
                     __LINE__);                                                              \
      return MD_ECUDA;                                                                       \
    }                                                                                        \
  } while (0)

constexpr int kWarp = 32;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Four-wide position record (x, y, z, unused) in the arithmetic type of the
// pair path: float4 in the mixed form, two 16-byte halves in FP64.
template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  using type = float4;
  __device__ __forceinline__ static float4 load(const float4 *p) { return __ldg(p); }
  __device__ __forceinline__ static void store(float4 *p, float x, float y, float z, float w = 0.f) {
    *p = make_float4(x, y, z, w);
  }
};
struct alignas(16) dvec4 {
  double x, y, z, w;
};
template <>
struct Vec4<double> {
  using type = dvec4;
  __device__ __forceinline__ static dvec4 load(const dvec4 *p) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
    double2 a = __ldg(q), b = __ldg(q + 1);
    return dvec4{a.x, a.y, b.x, b.y};
  }
  __device__ __forceinline__ static void store(dvec4 *p, double x, double y, double z, double w = 0.0) {
    double2 *q = reinterpret_cast<double2 *>(p);
    q[0] = make_double2(x, y);
    q[1] = make_double2(z, w);
  }
};

// 1/x for the FP32 pair terms: the hardware approximation (within one ulp),
// whose error (~1e-7 relative) is far below the FP32 rounding of the pair
// distance that the mixed-form force tolerance already covers.
__device__ __forceinline__ float pair_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double pair_rcp(double x) { return 1.0 / x; }

// Double-float numbers: an unevaluated sum h + l of two FP32 words with
// |l| <= ulp(h)/2 (about 48 significant bits).  GB300 runs FP64 at a small
// fraction of its FP32 rate, so the mixed form carries positions and
// velocities this way.  Built from the classical error-free transformations
// (Knuth's TwoSum, Dekker's FastTwoSum, the FMA form of Dekker's TwoProduct);
// the code is compiled without fast-math, so the compiler neither
// re-associates these sums nor flushes the small low words.
struct dfloat {
  float h, l;
};

__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {  // needs |a| >= |b|
  const float s = a + b;
  return dfloat{s, b - (s - a)};
}
__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return dfloat{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
  dfloat s = df_two_sum(a.h, b.h);
  const dfloat t = df_two_sum(a.l, b.l);
  s.l += t.h;
  s = df_fast_two_sum(s.h, s.l);
  s.l += t.l;
  return df_fast_two_sum(s.h, s.l);
}
__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ dfloat df_mul_f(dfloat a, float b) {
  const float p = a.h * b;
  float e = fmaf(a.h, b, -p);
  e = fmaf(a.l, b, e);
  return df_fast_two_sum(p, e);
}
// Products left unnormalised (p + e, |e| << |p|) and a compensated
// accumulator for them: the running sum s carries the rounded total and c
// the sum of every rounding error (TwoSum) and low part, so the value
// s + c keeps about 48 significant bits over a few dozen terms (the
// cascaded summation of Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005).
__device__ __forceinline__ dfloat df_prod(dfloat a, dfloat b) {  // unnormalised a * b
  const float p = a.h * b.h;
  return dfloat{p, fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p)))};
}
__device__ __forceinline__ dfloat df_prod_f(float a, dfloat b) {  // unnormalised a * b
  const float p = a * b.h;
  return dfloat{p, fmaf(a, b.l, fmaf(a, b.h, -p))};
}
struct dfacc {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(dfloat x) {
    const dfloat t = df_two_sum(s, x.h);
    s = t.h;
    c += t.l + x.l;
  }
  __device__ __forceinline__ void add(float x) {
    const dfloat t = df_two_sum(s, x);
    s = t.h;
    c += t.l;
  }
  // adds another accumulator (s2, c2)
  __device__ __forceinline__ void merge(float s2, float c2) {
    const dfloat t = df_two_sum(s, s2);
    s = t.h;
    c += t.l + c2;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Host / FP64 conversions (used at set-up and output only).
__host__ __device__ __forceinline__ dfloat df_from_double(double x) {
  const float h = (float)x;
  return dfloat{h, (float)(x - (double)h)};
}
__host__ __device__ __forceinline__ double df_to_double(dfloat a) { return (double)a.h + (double)a.l; }

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace otf
