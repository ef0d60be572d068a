// Multiple-tau correlator kernels and the corr_* C ABI
// (arXiv 2503.07526, Sec. 2.2; Appendix D Algorithms 1 and 2).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "corr.cuh"
#include "gk_tail.h"

namespace otf {

namespace {

constexpr int kPushThreads = 256;
constexpr int kPushWarps = kPushThreads / kWarp;

// Per-series correlators: one thread runs Algorithm 1 for one series.
template <typename T, typename Tin>
__global__ void k_push_series(CorrDev c, const Tin *__restrict__ x, const Tin *__restrict__ y,
                              PushIdx pi) {
  int64_t t;
  if (!resolve_push(pi, &t)) return;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < c.ns;
       s += (int64_t)gridDim.x * blockDim.x) {
    const T xv = (T)x[s];
    const T yv = c.cross ? (T)y[s] : xv;
    push_one_series<T>(c, s, xv, yv, t);
  }
}

// Vector access of V consecutive elements (16-byte aligned when V > 1).
template <typename E, int V>
struct VecIO {
  __device__ __forceinline__ static void load(const E *p, E *o) {
#pragma unroll
    for (int q = 0; q < V; ++q) o[q] = p[q];
  }
  __device__ __forceinline__ static void store(E *p, const E *v) {
#pragma unroll
    for (int q = 0; q < V; ++q) p[q] = v[q];
  }
};
template <>
struct VecIO<float, 4> {
  __device__ __forceinline__ static void load(const float *p, float *o) {
    const float4 a = *reinterpret_cast<const float4 *>(p);
    o[0] = a.x, o[1] = a.y, o[2] = a.z, o[3] = a.w;
  }
  __device__ __forceinline__ static void store(float *p, const float *v) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct VecIO<double, 2> {
  __device__ __forceinline__ static void load(const double *p, double *o) {
    const double2 a = *reinterpret_cast<const double2 *>(p);
    o[0] = a.x, o[1] = a.y;
  }
  __device__ __forceinline__ static void store(double *p, const double *v) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
  }
};
template <>
struct VecIO<double, 4> {
  __device__ __forceinline__ static void load(const double *p, double *o) {
    VecIO<double, 2>::load(p, o);
    VecIO<double, 2>::load(p + 2, o + 2);
  }
};

// Input samples of V series, converted to the ring type.
template <typename T, typename Tin, int V, bool VIN>
__device__ __forceinline__ void load_input(const Tin *p, T *o) {
  Tin a[V];
  if (VIN)
    VecIO<Tin, V>::load(p, a);
  else
#pragma unroll
    for (int q = 0; q < V; ++q) a[q] = p[q];
#pragma unroll
  for (int q = 0; q < V; ++q) o[q] = (T)a[q];
}

constexpr int kLoadsInFlight = 8;  // ring vectors loaded together per thread

// Grouped correlators (e.g. the per-atom velocity autocorrelation).  Thread
// (cx, g, tid) owns U vectors of V consecutive series, s = g gs +
// (cx blockDim + tid) U V, for good (so the per-block partial sums are
// deterministic), and each push is a pure stream: for every block the push
// reaches, the thread stores the new sample and loads the older ring vectors
// of kLoadsInFlight / U lags at a time (16-byte loads, one plane per lag:
// coalesced across the warp), forms the lag products in the ring type (FP32
// in the mixed form), sums them over its U V series and the warp with
// shuffles, then the CTA adds the FP64 sum over its warps into its own row
// of partial lag sums.  Two vectors per thread halve the shuffle reductions
// per byte streamed.  VIN: the input is 16-byte aligned and can be read as
// vectors.
template <typename T, typename Tin, int V, bool VIN, int U>
__global__ void __launch_bounds__(kPushThreads)
    k_push_grouped(CorrDev c, const Tin *__restrict__ x, const Tin *__restrict__ y, PushIdx pi) {
  constexpr int kLC = kLoadsInFlight / U;  // lags per load batch
  int64_t t;
  if (!resolve_push(pi, &t)) return;
  __shared__ double red[kPushWarps][64];
  const int g = blockIdx.y, cx = blockIdx.x;
  const int lane = threadIdx.x & (kWarp - 1), warp = threadIdx.x / kWarp;
  const int64_t i0 = ((int64_t)cx * blockDim.x + threadIdx.x) * U * V;  // index within the group
  const bool act = i0 < c.gs;
  const int64_t s = (int64_t)g * c.gs + (act ? i0 : 0);
  const int64_t plane = c.ns;
  T *rx = static_cast<T *>(c.ringx);
  T *ry = c.cross ? static_cast<T *>(c.ringy) : rx;
  int64_t Mk = 1;
  for (int k = 0; k < c.b; ++k) {
    if (k > 0) {
      Mk *= c.m;
      if (t % Mk) break;
    }
    const int64_t nk = t / Mk;
    const int slot = (int)((nk - 1) % c.p);
    const int lo = (k == 0) ? 0 : c.p / c.m;
    const int nl = (int)min((int64_t)c.p - 1, nk - 1) - lo + 1;
    T *rxk = rx + (int64_t)k * c.p * plane;
    T xk[U][V], yk[U][V];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int q = 0; q < V; ++q) xk[u][q] = yk[u][q] = T(0);
    if (act) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t su = s + u * V;
        if (k == 0) {
          load_input<T, Tin, V, VIN>(x + su, xk[u]);
          if (c.cross) load_input<T, Tin, V, VIN>(y + su, yk[u]);
        } else {
          // block k's sample: mean of block k-1's last m samples, oldest first
          const int64_t nprev = nk * c.m;
          const T *rp = rx + (int64_t)(k - 1) * c.p * plane;
          const T *rq = ry + (int64_t)(k - 1) * c.p * plane;
          T sx[V], sy[V], av[V];
#pragma unroll
          for (int q = 0; q < V; ++q) sx[q] = sy[q] = T(0);
          for (int j = c.m - 1; j >= 0; --j) {
            const int sl = (int)((nprev - 1 - j) % c.p);
            VecIO<T, V>::load(rp + sl * plane + su, av);
#pragma unroll
            for (int q = 0; q < V; ++q) sx[q] += av[q];
            if (c.cross) {
              VecIO<T, V>::load(rq + sl * plane + su, av);
#pragma unroll
              for (int q = 0; q < V; ++q) sy[q] += av[q];
            }
          }
#pragma unroll
          for (int q = 0; q < V; ++q) {
            xk[u][q] = sx[q] / T(c.m);
            yk[u][q] = sy[q] / T(c.m);
          }
        }
        if (!c.cross)
#pragma unroll
          for (int q = 0; q < V; ++q) yk[u][q] = xk[u][q];
        VecIO<T, V>::store(rxk + slot * plane + su, xk[u]);
        if (c.cross) VecIO<T, V>::store(ry + (int64_t)k * c.p * plane + slot * plane + su, yk[u]);
      }
    }
    for (int l0 = 0; l0 < nl; l0 += kLC) {
      T older[kLC][U][V];
#pragma unroll
      for (int l = 0; l < kLC; ++l) {
        const int lag = lo + l0 + l;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (act && l0 + l < nl) {
            if (lag == 0) {
#pragma unroll
              for (int q = 0; q < V; ++q) older[l][u][q] = xk[u][q];
            } else {
              int j = slot - lag;
              if (j < 0) j += c.p;
              VecIO<T, V>::load(rxk + j * plane + s + u * V, older[l][u]);
            }
          } else {
#pragma unroll
            for (int q = 0; q < V; ++q) older[l][u][q] = T(0);
          }
        }
      }
#pragma unroll
      for (int l = 0; l < kLC; ++l) {
        if (l0 + l < nl) {
          T a = T(0);
#pragma unroll
          for (int u = 0; u < U; ++u)
#pragma unroll
            for (int q = 0; q < V; ++q) a += older[l][u][q] * yk[u][q];
          a = warp_sum(a);
          if (lane == 0) red[warp][l0 + l] = (double)a;
        }
      }
    }
    if (nl <= 0) continue;  // uniform over the grid
    __syncthreads();
    if (threadIdx.x < nl) {
      double sum = 0.0;
      for (int w = 0; w < kPushWarps; ++w) sum += red[w][threadIdx.x];
      c.vals[(((int64_t)g * c.nchunk + cx) * c.b + k) * c.p + lo + threadIdx.x] += sum;
    }
    __syncthreads();
  }
}

// Sums the per-block partial lag sums of each group in a fixed order.
__global__ void k_fold(CorrDev c, double *__restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)c.b * c.p;
  if (e >= c.ng * per) return;
  const int64_t g = e / per, kl = e % per;
  double s = 0.0;
  for (int cx = 0; cx < c.nchunk; ++cx) s += c.vals[(g * c.nchunk + cx) * per + kl];
  out[e] = s;
}

template <typename T, typename Tin>
int launch_grouped(const CorrDev &c, const Tin *x, const Tin *y, PushIdx pi, cudaStream_t s) {
  dim3 grid(c.nchunk, (unsigned)c.ng);
  constexpr int V = 16 / sizeof(T);
  if (c.vec == V) {
    const bool vin = (reinterpret_cast<uintptr_t>(x) % (V * sizeof(Tin)) == 0) &&
                     (!c.cross || reinterpret_cast<uintptr_t>(y) % (V * sizeof(Tin)) == 0);
    if (c.vu == 2) {
      if (vin)
        k_push_grouped<T, Tin, V, true, 2><<<grid, kPushThreads, 0, s>>>(c, x, y, pi);
      else
        k_push_grouped<T, Tin, V, false, 2><<<grid, kPushThreads, 0, s>>>(c, x, y, pi);
    } else if (vin) {
      k_push_grouped<T, Tin, V, true, 1><<<grid, kPushThreads, 0, s>>>(c, x, y, pi);
    } else {
      k_push_grouped<T, Tin, V, false, 1><<<grid, kPushThreads, 0, s>>>(c, x, y, pi);
    }
  } else {
    k_push_grouped<T, Tin, 1, false, 1><<<grid, kPushThreads, 0, s>>>(c, x, y, pi);
  }
  OTF_LAUNCH_CHECK();
  return MD_OK;
}

// Time-blocked pushes of a grouped autocorrelator (the per-atom velocity
// correlator of an MD run), block 0: the pushes done+1 .. t (at most
// bi.block) in one pass, with the same series-to-thread map as
// k_push_grouped (U vectors of V series per thread).  The thread loads the
// p-1 most recent ring samples of its series once, keeps them and the new
// samples in registers, forms every lag product of every new push from them
// and stores only the new samples, so a block of pushes reads the ring once
// instead of once per push.  Its lag sums are summed over the new pushes and
// the thread's series before the warp and CTA sums.  Products and lags are
// those of Algorithm 1; only the order of the additions within a lag sum
// differs.  k_push_higher then applies the higher blocks.
template <typename T, typename Tin, int V, bool VIN, int U>
__global__ void __launch_bounds__(kPushThreads, sizeof(T) == 4 ? 2 : 1)
    k_push_block0(CorrDev c, const Tin *__restrict__ xh, BlockIdx bi) {
  constexpr int P1 = 15;  // older samples kept for block 0 (p - 1 with p = 16)
  const int64_t st = *bi.d_step - *bi.d_base;
  const int64_t t = (bi.u > 0 && st > 0) ? st / bi.u : 0;
  const int64_t done = *bi.d_done;
  const int nnew = (int)(t - done);
  if (nnew > bi.block) {  // a pass was lost: report it instead of dropping pushes silently
    if (bi.d_err && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) atomicOr(bi.d_err, ERR_PUSH_BACKLOG);
    return;
  }
  if (nnew <= 0 || (!bi.flush && nnew < bi.block)) return;
  __shared__ double red[kPushWarps][64];
  const int g = blockIdx.y, cx = blockIdx.x;
  const int lane = threadIdx.x & (kWarp - 1), warp = threadIdx.x / kWarp;
  const int64_t i0 = ((int64_t)cx * blockDim.x + threadIdx.x) * U * V;
  const bool act = i0 < c.gs;
  const int64_t s = (int64_t)g * c.gs + (act ? i0 : 0);
  const int64_t plane = c.ns;
  T *rx = static_cast<T *>(c.ringx);

  // block 0 over the new pushes, one vector of series at a time
  T acc0[P1 + 1];
#pragma unroll
  for (int l = 0; l <= P1; ++l) acc0[l] = T(0);
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t su = s + u * V;
    T win[P1][V];  // win[l]: the sample of push done - l
#pragma unroll
    for (int l = 0; l < P1; ++l) {
      if (act && l < c.p - 1 && done - l >= 1) {
        VecIO<T, V>::load(rx + ((done - l - 1) % c.p) * plane + su, win[l]);
      } else {
#pragma unroll
        for (int q = 0; q < V; ++q) win[l][q] = T(0);
      }
    }
    T xn[kPushBlock][V];
#pragma unroll
    for (int j = 0; j < kPushBlock; ++j) {
      if (act && j < nnew)
        load_input<T, Tin, V, VIN>(xh + ((done + j) % kPushBlock) * plane + su, xn[j]);
      else
#pragma unroll
        for (int q = 0; q < V; ++q) xn[j][q] = T(0);
    }
#pragma unroll
    for (int j = 0; j < kPushBlock; ++j) {
      if (j < nnew) {
        const int64_t tp = done + 1 + j;  // this push
        if (act) VecIO<T, V>::store(rx + ((tp - 1) % c.p) * plane + su, xn[j]);
#pragma unroll
        for (int l = 0; l <= P1; ++l) {
          if (l < c.p && tp - l >= 1) {  // a lag of this block whose older sample exists
            T a = T(0);
#pragma unroll
            for (int q = 0; q < V; ++q) {
              const T o = (l <= j) ? xn[j - l][q] : win[l - j - 1 < P1 ? l - j - 1 : 0][q];
              a += o * xn[j][q];
            }
            acc0[l] += a;
          }
        }
      }
    }
  }
#pragma unroll
  for (int l = 0; l <= P1; ++l) {
    const T a = warp_sum(acc0[l]);
    if (lane == 0) red[warp][l] = (double)a;
  }
  __syncthreads();
  if (threadIdx.x <= P1 && (int)threadIdx.x < c.p) {
    double sum = 0.0;
    for (int w = 0; w < kPushWarps; ++w) sum += red[w][threadIdx.x];
    c.vals[(((int64_t)g * c.nchunk + cx) * c.b + 0) * c.p + threadIdx.x] += sum;
  }
  __syncthreads();
}

// The higher blocks of the pushes done+1 .. t that k_push_block0 applied to
// block 0, push by push and block by block as in k_push_grouped (block k's
// sample is the mean of block k-1's last m samples, already stored); the
// last CTA to finish records the pushes as applied.
template <typename T, int V, int U>
__global__ void __launch_bounds__(kPushThreads) k_push_higher(CorrDev c, BlockIdx bi) {
  const int64_t st = *bi.d_step - *bi.d_base;
  const int64_t t = (bi.u > 0 && st > 0) ? st / bi.u : 0;
  const int64_t done = *bi.d_done;
  const int nnew = (int)(t - done);
  if (nnew > bi.block) {  // a pass was lost: report it instead of dropping pushes silently
    if (bi.d_err && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) atomicOr(bi.d_err, ERR_PUSH_BACKLOG);
    return;
  }
  if (nnew <= 0 || (!bi.flush && nnew < bi.block)) return;
  __shared__ double red[kPushWarps][64];
  const int g = blockIdx.y, cx = blockIdx.x;
  const int lane = threadIdx.x & (kWarp - 1), warp = threadIdx.x / kWarp;
  const int64_t i0 = ((int64_t)cx * blockDim.x + threadIdx.x) * U * V;
  const bool act = i0 < c.gs;
  const int64_t s = (int64_t)g * c.gs + (act ? i0 : 0);
  const int64_t plane = c.ns;
  T *rx = static_cast<T *>(c.ringx);
  // higher blocks, push by push
  for (int j = 0; j < nnew; ++j) {
    const int64_t tp = done + 1 + j;
    int64_t Mk = 1;
    for (int k = 1; k < c.b; ++k) {
      Mk *= c.m;
      if (tp % Mk) break;
      const int64_t nk = tp / Mk;
      const int slot = (int)((nk - 1) % c.p);
      const int lo = c.p / c.m;
      const int nl = (int)min((int64_t)c.p - 1, nk - 1) - lo + 1;
      T *rxk = rx + (int64_t)k * c.p * plane;
      T xk[U][V];
#pragma unroll
      for (int u = 0; u < U; ++u) {
#pragma unroll
        for (int q = 0; q < V; ++q) xk[u][q] = T(0);
        if (act) {
          const int64_t su = s + u * V;
          const int64_t nprev = nk * c.m;
          const T *rp = rx + (int64_t)(k - 1) * c.p * plane;
          T sx[V], av[V];
#pragma unroll
          for (int q = 0; q < V; ++q) sx[q] = T(0);
          for (int jj = c.m - 1; jj >= 0; --jj) {
            const int sl = (int)((nprev - 1 - jj) % c.p);
            VecIO<T, V>::load(rp + sl * plane + su, av);
#pragma unroll
            for (int q = 0; q < V; ++q) sx[q] += av[q];
          }
#pragma unroll
          for (int q = 0; q < V; ++q) xk[u][q] = sx[q] / T(c.m);
          VecIO<T, V>::store(rxk + slot * plane + su, xk[u]);
        }
      }
      for (int l = 0; l < nl; ++l) {
        const int lag = lo + l;
        int jr = slot - lag;
        if (jr < 0) jr += c.p;
        T a = T(0);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          T older[V];
          if (act) {
            VecIO<T, V>::load(rxk + jr * plane + s + u * V, older);
          } else {
#pragma unroll
            for (int q = 0; q < V; ++q) older[q] = T(0);
          }
#pragma unroll
          for (int q = 0; q < V; ++q) a += older[q] * xk[u][q];
        }
        a = warp_sum(a);
        if (lane == 0) red[warp][l] = (double)a;
      }
      if (nl <= 0) continue;
      __syncthreads();
      if (threadIdx.x < nl) {
        double sum = 0.0;
        for (int w = 0; w < kPushWarps; ++w) sum += red[w][threadIdx.x];
        c.vals[(((int64_t)g * c.nchunk + cx) * c.b + k) * c.p + lo + threadIdx.x] += sum;
      }
      __syncthreads();
    }
  }

  // the last CTA to finish records the pushes as applied
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(bi.d_ctas, 1u) == gridDim.x * gridDim.y - 1) {
      *bi.d_done = t;
      *bi.d_ctas = 0u;
      __threadfence();
    }
  }
}

template <typename T, typename Tin>
int launch_grouped_block(const CorrDev &c, const Tin *x, BlockIdx bi, cudaStream_t s) {
  dim3 grid(c.nchunk, (unsigned)c.ng);
  constexpr int V = 16 / sizeof(T);
  if (c.vec == V) {
    const bool vin = reinterpret_cast<uintptr_t>(x) % (V * sizeof(Tin)) == 0 &&
                     (c.ns * sizeof(Tin)) % (V * sizeof(Tin)) == 0;
    if (c.vu == 2) {
      if (vin)
        k_push_block0<T, Tin, V, true, 2><<<grid, kPushThreads, 0, s>>>(c, x, bi);
      else
        k_push_block0<T, Tin, V, false, 2><<<grid, kPushThreads, 0, s>>>(c, x, bi);
      k_push_higher<T, V, 2><<<grid, kPushThreads, 0, s>>>(c, bi);
    } else {
      if (vin)
        k_push_block0<T, Tin, V, true, 1><<<grid, kPushThreads, 0, s>>>(c, x, bi);
      else
        k_push_block0<T, Tin, V, false, 1><<<grid, kPushThreads, 0, s>>>(c, x, bi);
      k_push_higher<T, V, 1><<<grid, kPushThreads, 0, s>>>(c, bi);
    }
  } else {
    k_push_block0<T, Tin, 1, false, 1><<<grid, kPushThreads, 0, s>>>(c, x, bi);
    k_push_higher<T, 1, 1><<<grid, kPushThreads, 0, s>>>(c, bi);
  }
  OTF_LAUNCH_CHECK();
  return MD_OK;
}

template <typename T, typename Tin>
int launch_series(const CorrDev &c, const Tin *x, const Tin *y, PushIdx pi, cudaStream_t s) {
  int blocks = std::max(1, std::min(ceil_div(c.ns, 128), 152 * 8));
  k_push_series<T, Tin><<<blocks, 128, 0, s>>>(c, x, y, pi);
  OTF_LAUNCH_CHECK();
  return MD_OK;
}

}  // namespace

int validate_corr_params(const corr_params &p) {
  if (p.b < 1 || p.b > 32 || p.p < 2 || p.p > 64 || p.m < 1 || p.m > p.p || p.p % p.m != 0) {
    set_error("correlator needs 1 <= b <= 32, 2 <= p <= 64, 1 <= m <= p, m | p (got b=%d p=%d m=%d)",
              p.b, p.p, p.m);
    return MD_EINVAL;
  }
  if (p.nseries < 1 || p.group_size < 1 || p.nseries % p.group_size != 0) {
    set_error("nseries must be a positive multiple of group_size");
    return MD_EINVAL;
  }
  if (p.precision != MD_PREC_FP64 && p.precision != MD_PREC_MIXED) {
    set_error("unknown precision %d", p.precision);
    return MD_EINVAL;
  }
  if (!(p.dt_unit > 0.0)) {
    set_error("dt_unit must be positive");
    return MD_EINVAL;
  }
  return MD_OK;
}

int Correlator::create(const corr_params &p, cudaStream_t s, cudaStream_t zero_on) {
  int rc = validate_corr_params(p);
  if (rc) return rc;
  prm = p;
  prec = p.precision;
  stream = s;
  grouped = p.group_size > 1;
  dev.b = p.b;
  dev.p = p.p;
  dev.m = p.m;
  dev.cross = p.cross ? 1 : 0;
  dev.ns = p.nseries;
  dev.gs = p.group_size;
  dev.ng = p.nseries / p.group_size;
  if (grouped) {
    // one 16-byte vector of series per thread when the group size allows it
    const int vw = (int)(16 / (p.precision == MD_PREC_FP64 ? sizeof(double) : sizeof(float)));
    dev.vec = (dev.gs % vw == 0) ? vw : 1;
    // two vectors per thread when the group splits evenly into them
    dev.vu = (dev.vec == vw && dev.gs % (2 * vw) == 0) ? 2 : 1;
    const int64_t per_block = (int64_t)kPushThreads * dev.vec * dev.vu;
    dev.nchunk = (int)((dev.gs + per_block - 1) / per_block);
  } else {
    dev.vec = 1;
    dev.vu = 1;
    dev.nchunk = 1;
  }
  const size_t esz = prec == MD_PREC_FP64 ? sizeof(double) : sizeof(float);
  const size_t ring = (size_t)p.b * p.p * p.nseries * esz;
  OTF_CUDA(cudaMalloc(&dev.ringx, ring));
  if (dev.cross) OTF_CUDA(cudaMalloc(&dev.ringy, ring));
  const size_t nvals = grouped ? (size_t)dev.ng * dev.nchunk * p.b * p.p : (size_t)p.nseries * p.b * p.p;
  OTF_CUDA(cudaMalloc(&dev.vals, nvals * sizeof(double)));
  OTF_CUDA(cudaMalloc(&d_fold, (size_t)dev.ng * p.b * p.p * sizeof(double)));
  return reset(zero_on);
}

int Correlator::reset(cudaStream_t on) {
  cudaStream_t zs = on ? on : stream;
  const size_t esz = prec == MD_PREC_FP64 ? sizeof(double) : sizeof(float);
  const size_t ring = (size_t)prm.b * prm.p * prm.nseries * esz;
  const size_t nvals = grouped ? (size_t)dev.ng * dev.nchunk * prm.b * prm.p : (size_t)prm.nseries * prm.b * prm.p;
  OTF_CUDA(cudaMemsetAsync(dev.ringx, 0, ring, zs));
  if (dev.cross) OTF_CUDA(cudaMemsetAsync(dev.ringy, 0, ring, zs));
  OTF_CUDA(cudaMemsetAsync(dev.vals, 0, nvals * sizeof(double), zs));
  pushes = 0;
  return MD_OK;
}

void Correlator::destroy() {
  cudaFree(dev.ringx);
  if (dev.ringy) cudaFree(dev.ringy);
  cudaFree(dev.vals);
  cudaFree(d_fold);
  cudaFree(d_in);
  dev.ringx = dev.ringy = nullptr;
  dev.vals = d_fold = d_in = nullptr;
}

int Correlator::launch_push(const void *x, const void *y, bool input_fp32, PushIdx pi, cudaStream_t s) {
  const bool fp64 = prec == MD_PREC_FP64;
  if (grouped) {
    if (fp64) {
      if (input_fp32) return launch_grouped<double, float>(dev, (const float *)x, (const float *)y, pi, s);
      return launch_grouped<double, double>(dev, (const double *)x, (const double *)y, pi, s);
    }
    if (input_fp32) return launch_grouped<float, float>(dev, (const float *)x, (const float *)y, pi, s);
    return launch_grouped<float, double>(dev, (const double *)x, (const double *)y, pi, s);
  }
  if (fp64) {
    if (input_fp32) return launch_series<double, float>(dev, (const float *)x, (const float *)y, pi, s);
    return launch_series<double, double>(dev, (const double *)x, (const double *)y, pi, s);
  }
  if (input_fp32) return launch_series<float, float>(dev, (const float *)x, (const float *)y, pi, s);
  return launch_series<float, double>(dev, (const double *)x, (const double *)y, pi, s);
}

int Correlator::launch_push_block(const void *x, bool input_fp32, BlockIdx bi, cudaStream_t s) {
  if (!grouped || dev.cross || prm.p > 16 || bi.block < 1 || bi.block > kPushBlock) {
    set_error("blocked pushes need a grouped autocorrelator with p <= 16 and 1..%d pushes per block", kPushBlock);
    return MD_EINVAL;
  }
  if (prec == MD_PREC_FP64) {
    if (input_fp32) return launch_grouped_block<double, float>(dev, (const float *)x, bi, s);
    return launch_grouped_block<double, double>(dev, (const double *)x, bi, s);
  }
  if (input_fp32) return launch_grouped_block<float, float>(dev, (const float *)x, bi, s);
  return launch_grouped_block<float, double>(dev, (const double *)x, bi, s);
}

int Correlator::fetch(double *vals_host) {
  if (before_read) {
    const int rc = before_read(read_ctx);
    if (rc) return rc;
  }
  const size_t n = (size_t)dev.ng * prm.b * prm.p;
  const double *src = dev.vals;
  if (grouped) {
    k_fold<<<ceil_div((int64_t)n, 256), 256, 0, stream>>>(dev, d_fold);
    OTF_LAUNCH_CHECK();
    src = d_fold;
  }
  OTF_CUDA(cudaMemcpyAsync(vals_host, src, n * sizeof(double), cudaMemcpyDeviceToHost, stream));
  OTF_CUDA(cudaStreamSynchronize(stream));
  return MD_OK;
}

}  // namespace otf

using otf::Correlator;
using otf::set_error;

namespace {

// Products per series at each (block, lag) after t pushes, and blocks used.
void counts_from_pushes(const corr_params &p, int64_t t, std::vector<int64_t> &count, int *used) {
  count.assign((size_t)p.b * p.p, 0);
  *used = 0;
  int64_t Mk = 1;
  for (int k = 0; k < p.b; ++k) {
    if (k > 0) Mk *= p.m;
    const int64_t nk = t / Mk;
    if (nk < 1) break;
    *used = k + 1;
    const int lo = (k == 0) ? 0 : p.p / p.m;
    for (int lag = lo; lag < p.p; ++lag) count[(size_t)k * p.p + lag] = std::max<int64_t>(0, nk - lag);
  }
}

}  // namespace

extern "C" {

int corr_create(const corr_params *cp, void *cuda_stream, corr_handle **out) {
  otf::clear_error();
  if (!cp || !out) {
    set_error("corr_create: null argument");
    return MD_EINVAL;
  }
  *out = nullptr;
  corr_handle *h = new (std::nothrow) corr_handle;
  if (!h) return MD_ENOMEM;
  int rc = h->c.create(*cp, (cudaStream_t)cuda_stream);
  if (rc) {
    h->c.destroy();
    delete h;
    return rc;
  }
  rc = [&]() -> int {
    OTF_CUDA(cudaMalloc(&h->c.d_in, sizeof(double) * 2 * cp->nseries));
    return MD_OK;
  }();
  if (rc) {
    h->c.destroy();
    delete h;
    return rc;
  }
  *out = h;
  return MD_OK;
}

int corr_push(corr_handle *h, const double *x, const double *y, int64_t nseries, int32_t mem) {
  otf::clear_error();
  if (!h || !x) {
    set_error("corr_push: null argument");
    return MD_EINVAL;
  }
  Correlator &c = h->c;
  if (c.borrowed) {
    set_error("corr_push: this correlator is fed by md_step");
    return MD_EINVAL;
  }
  if (nseries != c.prm.nseries) {
    set_error("corr_push: %lld series given, correlator has %lld", (long long)nseries,
              (long long)c.prm.nseries);
    return MD_EINVAL;
  }
  if (c.prm.cross && !y) {
    set_error("corr_push: cross correlator needs y");
    return MD_EINVAL;
  }
  const double *dx = x, *dy = y;
  if (mem == MD_MEM_HOST) {
    OTF_CUDA(cudaMemcpyAsync(c.d_in, x, sizeof(double) * nseries, cudaMemcpyHostToDevice, c.stream));
    dx = c.d_in;
    if (c.prm.cross) {
      OTF_CUDA(cudaMemcpyAsync(c.d_in + nseries, y, sizeof(double) * nseries, cudaMemcpyHostToDevice, c.stream));
      dy = c.d_in + nseries;
    }
    // host buffers may be reused as soon as the call returns
    OTF_CUDA(cudaStreamSynchronize(c.stream));
  } else if (mem != MD_MEM_DEVICE) {
    set_error("corr_push: mem must be MD_MEM_HOST or MD_MEM_DEVICE");
    return MD_EINVAL;
  }
  c.pushes += 1;
  otf::PushIdx pi{nullptr, nullptr, 1, c.pushes};
  int rc = c.launch_push(dx, c.prm.cross ? dy : dx, false, pi, c.stream);
  if (rc) c.pushes -= 1;
  return rc;
}

int corr_raw(corr_handle *h, double *values, int64_t *count, int32_t *blocks_used) {
  otf::clear_error();
  if (!h) {
    set_error("corr_raw: null handle");
    return MD_EINVAL;
  }
  Correlator &c = h->c;
  std::vector<double> v((size_t)c.dev.ng * c.prm.b * c.prm.p);
  int rc = c.fetch(v.data());
  if (rc) return rc;
  std::vector<int64_t> cnt;
  int used = 0;
  counts_from_pushes(c.prm, c.push_count(), cnt, &used);
  if (values) std::memcpy(values, v.data(), sizeof(double) * v.size());
  if (count) std::memcpy(count, cnt.data(), sizeof(int64_t) * cnt.size());
  if (blocks_used) *blocks_used = used;
  return MD_OK;
}

int corr_read(corr_handle *h, int64_t g, double *times, double *values, int64_t cap, int64_t *n) {
  otf::clear_error();
  if (!h || !n) {
    set_error("corr_read: null argument");
    return MD_EINVAL;
  }
  Correlator &c = h->c;
  const corr_params &p = c.prm;
  const int64_t ng = c.dev.ng;
  if (g < -1 || g >= ng) {
    set_error("corr_read: group %lld out of range", (long long)g);
    return MD_EINVAL;
  }
  std::vector<double> v((size_t)ng * p.b * p.p);
  int rc = c.fetch(v.data());
  if (rc) return rc;
  std::vector<int64_t> cnt;
  int used = 0;
  counts_from_pushes(p, c.push_count(), cnt, &used);
  // Algorithm 2: block 1 lags 0..p-1, then blocks 2..used lags p/m..p-1.
  int64_t npts = 0;
  double scale = 1.0;
  for (int k = 0; k < used; ++k) {
    if (k > 0) scale *= p.m;
    const int lo = (k == 0) ? 0 : p.p / p.m;
    for (int lag = lo; lag < p.p; ++lag) {
      const int64_t ct = cnt[(size_t)k * p.p + lag];
      if (ct <= 0) continue;
      if (npts < cap && times && values) {
        double sum = 0.0;
        if (g >= 0) {
          sum = v[((size_t)g * p.b + k) * p.p + lag];
        } else {
          for (int64_t gg = 0; gg < ng; ++gg) sum += v[((size_t)gg * p.b + k) * p.p + lag];
          sum /= (double)ng;
        }
        times[npts] = lag * scale * p.dt_unit;
        values[npts] = sum / ((double)ct * (double)p.group_size);
      }
      ++npts;
    }
  }
  *n = npts;
  if (npts > cap) {
    set_error("corr_read: %lld points need a larger buffer", (long long)npts);
    return MD_ECAP;
  }
  return MD_OK;
}

int corr_read_rows(corr_handle *h, int64_t g0, int64_t rows, int64_t avg, double *times, double *values,
                   int64_t cap, int64_t *n) {
  otf::clear_error();
  if (!h || !n || rows < 1 || avg < 1) {
    set_error("corr_read_rows: null argument or rows / avg < 1");
    return MD_EINVAL;
  }
  Correlator &c = h->c;
  const corr_params &p = c.prm;
  const int64_t ng = c.dev.ng;
  if (g0 < 0 || g0 + rows * avg > ng) {
    set_error("corr_read_rows: groups %lld..%lld out of range (%lld groups)", (long long)g0,
              (long long)(g0 + rows * avg - 1), (long long)ng);
    return MD_EINVAL;
  }
  std::vector<double> v((size_t)ng * p.b * p.p);
  int rc = c.fetch(v.data());
  if (rc) return rc;
  std::vector<int64_t> cnt;
  int used = 0;
  counts_from_pushes(p, c.push_count(), cnt, &used);
  // the Algorithm 2 grid, as in corr_read, for every row at once
  int64_t npts = 0;
  double scale = 1.0;
  for (int k = 0; k < used; ++k) {
    if (k > 0) scale *= p.m;
    const int lo = (k == 0) ? 0 : p.p / p.m;
    for (int lag = lo; lag < p.p; ++lag) {
      const int64_t ct = cnt[(size_t)k * p.p + lag];
      if (ct <= 0) continue;
      if (npts < cap && times && values) {
        times[npts] = lag * scale * p.dt_unit;
        for (int64_t r = 0; r < rows; ++r) {
          double sum = 0.0;
          for (int64_t a = 0; a < avg; ++a) sum += v[((size_t)(g0 + r * avg + a) * p.b + k) * p.p + lag];
          values[r * cap + npts] = sum / (double)avg / ((double)ct * (double)p.group_size);
        }
      }
      ++npts;
    }
  }
  *n = npts;
  if (npts > cap) {
    set_error("corr_read_rows: %lld points need a larger buffer", (long long)npts);
    return MD_ECAP;
  }
  return MD_OK;
}

int corr_pushes(corr_handle *h, int64_t *n) {
  if (!h || !n) return MD_EINVAL;
  *n = h->c.push_count();
  return MD_OK;
}

int corr_reset(corr_handle *h) {
  otf::clear_error();
  if (!h) return MD_EINVAL;
  if (h->c.borrowed) {
    set_error("corr_reset: use md_reset_correlators for a system's correlators");
    return MD_EINVAL;
  }
  return h->c.reset();
}

void corr_free(corr_handle *h) {
  if (!h || h->c.borrowed) return;
  cudaStreamSynchronize(h->c.stream);
  h->c.destroy();
  delete h;
}

}  // extern "C"
