// Device-resident multiple-tau correlators (arXiv 2503.07526, Sec. 2.2 and
// Appendix D Algorithm 1).
//
// GB300 layout.  A correlator holds ns series that all receive a sample at
// the same pushes.  The ring of block k, slot j is one contiguous plane of ns
// values, ring[k][j][s], so every push streams coalesced planes.  Every
// per-level counter of Algorithm 1 (insert pointer, samples received,
// accumulator fill, products per lag) depends only on the number of pushes
// t, so it is derived from t instead of stored:
//   block k (0-based) receives a sample at push t iff m^k divides t;
//   it has then received n_k = t / m^k samples, the new one in slot
//   (n_k - 1) mod p;
//   the sample is the mean of the last m samples of block k-1, summed oldest
//   first (the accumulator of Algorithm 1, which holds exactly those m);
//   lags 0..p-1 on block 0, p/m..p-1 above, each formed when lag < n_k, so
//   count[k][lag] = max(0, n_k - lag).
// Lag products are the older x times the newer y (Sec. 2.2 Eq. (cor)).
#pragma once

#include "common.cuh"

namespace otf {

struct CorrDev {
  int b, p, m, cross;
  int64_t ns, gs, ng;  // series, series per group, groups
  int nchunk;          // blocks per group (grouped kernel)
  int vec;             // series per vector in the grouped kernel (1, 2 or 4)
  int vu;              // vectors per thread in the grouped kernel (1 or 2)
  void *ringx, *ringy; // [b][p][ns] of the ring type
  double *vals;        // per-series: [ns][b][p]; grouped: [ng][nchunk][b][p]
};

// Which push this is: from a device MD step counter (t = (step - base) / u,
// skipped unless u divides step - base) or a host count.
struct PushIdx {
  const int64_t *d_step;
  const int64_t *d_base;
  int64_t u;
  int64_t t_host;
};

// Time-blocked pushes of a grouped autocorrelator fed by an MD step: the
// sample of push t waits in input slot (t - 1) mod kPushBlock (each [ns])
// and the waiting pushes are applied in one pass once `block` of them wait
// (or whatever waits, when flushing): done+1 .. t, with t from the step
// counter as in PushIdx.  A block holds at most p - m + 1 pushes, so that
// its block-0 stores cannot overwrite a sample its first block-1 sample
// still needs.  The pass's last CTA advances *d_done.
constexpr int kPushBlock = 8;
struct BlockIdx {
  const int64_t *d_step;
  const int64_t *d_base;
  int64_t u;
  int64_t *d_done;   // pushes applied so far
  unsigned *d_ctas;  // CTAs of the current pass that have finished (returns to 0)
  int block;         // pushes per pass: min(kPushBlock, p - m + 1)
  int flush;         // 1: apply a partial block too
  unsigned *d_err;   // device error word (ERR_PUSH_BACKLOG), may be null
};

__device__ __forceinline__ bool resolve_push(const PushIdx &pi, int64_t *t) {
  if (pi.d_step) {
    const int64_t st = *pi.d_step - (pi.d_base ? *pi.d_base : 0);
    if (pi.u <= 0 || st <= 0 || st % pi.u) return false;
    *t = st / pi.u;
  } else {
    *t = pi.t_host;
  }
  return *t > 0;
}

// Algorithm 1 for one series s at push t, every block touched by this push;
// lag sums go straight into vals[s][k][lag] (per-series correlators).
template <typename T>
__device__ void push_one_series(const CorrDev &c, int64_t s, T xv, T yv, int64_t t) {
  T *rx = static_cast<T *>(c.ringx);
  T *ry = c.cross ? static_cast<T *>(c.ringy) : rx;
  const int64_t plane = c.ns;
  int64_t Mk = 1;
  for (int k = 0; k < c.b; ++k) {
    if (k > 0) {
      Mk *= c.m;
      if (t % Mk) break;
    }
    const int64_t nk = t / Mk;
    const int slot = (int)((nk - 1) % c.p);
    T xk = xv, yk = yv;
    if (k > 0) {
      const int64_t nprev = nk * c.m;
      T sx = T(0), sy = T(0);
      for (int j = c.m - 1; j >= 0; --j) {
        const int sl = (int)((nprev - 1 - j) % c.p);
        sx += rx[((int64_t)(k - 1) * c.p + sl) * plane + s];
        if (c.cross) sy += ry[((int64_t)(k - 1) * c.p + sl) * plane + s];
      }
      xk = sx / T(c.m);
      yk = c.cross ? sy / T(c.m) : xk;
    }
    rx[((int64_t)k * c.p + slot) * plane + s] = xk;
    if (c.cross) ry[((int64_t)k * c.p + slot) * plane + s] = yk;
    const int lo = (k == 0) ? 0 : c.p / c.m;
    const int hi = (int)min((int64_t)c.p - 1, nk - 1);
    double *vs = c.vals + (s * c.b + k) * c.p;
    for (int lag = lo; lag <= hi; ++lag) {
      int j = slot - lag;
      if (j < 0) j += c.p;
      const T older = (lag == 0) ? xk : rx[((int64_t)k * c.p + j) * plane + s];
      vs[lag] += (double)(older * yk);
    }
  }
}

// Host side of one correlator.
struct Correlator {
  corr_params prm{};
  int prec = MD_PREC_FP64;
  bool grouped = false;
  bool borrowed = false;   // owned by an MD system
  cudaStream_t stream = nullptr;
  CorrDev dev{};
  int64_t pushes = 0;      // free-standing: pushes so far
  const int64_t *host_steps = nullptr;  // MD-owned: host mirror of the step count
  const int64_t *host_base = nullptr;   // MD-owned: step of the last reset
  int64_t u = 1;           // MD-owned: steps per push
  int (*before_read)(void *) = nullptr;  // MD-owned: applies waiting pushes before a readout
  void *read_ctx = nullptr;
  double *d_in = nullptr;  // staging for host pushes, [2][ns]
  double *d_fold = nullptr;// [ng][b][p] folded lag sums

  // zero_on: the stream of the initial zeroing (null: s); a caller that
  // passes another stream orders s after it before the first push
  int create(const corr_params &p, cudaStream_t s, cudaStream_t zero_on = nullptr);
  void destroy();
  int reset(cudaStream_t on = nullptr);
  int64_t push_count() const {
    if (!host_steps) return pushes;
    return u > 0 ? (*host_steps - (host_base ? *host_base : 0)) / u : 0;
  }
  // Enqueues one push whose input already lives on the device.
  int launch_push(const void *x, const void *y, bool input_fp32, PushIdx pi, cudaStream_t s);
  // Enqueues the waiting pushes of a grouped autocorrelator whose samples sit
  // in kPushBlock slots of ns values at x (see BlockIdx).
  int launch_push_block(const void *x, bool input_fp32, BlockIdx bi, cudaStream_t s);
  // Lag sums [ng][b][p] on the host (folds the per-block partial sums).
  int fetch(double *vals_host);
};

// Copies host parameters with validation; returns MD_OK or MD_EINVAL.
int validate_corr_params(const corr_params &p);

}  // namespace otf

struct corr_handle_s {
  otf::Correlator c;
};
