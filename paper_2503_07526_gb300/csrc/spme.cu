// Smooth particle-mesh Ewald (Essmann et al. 1995; arXiv 2503.07526
// Sec. 5.3 and Appendix B) for the ionic-melt path.  Per step:
//   1. spread: every atom adds q M_n(u_x - k_x) M_n(u_y - k_y) M_n(u_z - k_z)
//      to the n^3 mesh points around it (fixed-point integer atomics, so
//      the sums do not depend on the order of the atoms: 64-bit words at a
//      scale of 2^40 in the mixed form, 128-bit words at 2^80 in FP64);
//   2. forward real-to-complex FFT of the mesh (cuFFT);
//   3. multiply by B(m) C(m) (phi mesh) and by B(m) C(m) h(m) (psi mesh),
//      C(m) = exp(-pi^2 m^2 / alpha^2) / (pi V m^2),
//      h(m) = 2 (1 + pi^2 m^2 / alpha^2) / m^2;
//   4. two inverse FFTs;
//   5. gather: each atom's spline weights, their first and second
//      derivatives read phi (energy, force) and psi (virial).
// Per atom j, with the sums over its n^3 mesh points:
//   E_j = 1/2 ke q_j sum W_j phi,  F_j = -ke q_j (K/L) sum grad_u W_j phi,
//   W_j,ab = delta_ab E_j + ke q_j K^2 / (8 pi^2 L^2) sum d_a d_b W_j psi,
// the last being Appendix B's form of the per-particle reciprocal virial
// (the factor m_a m_b of the k-space virial carried by two derivatives of
// the spline weights).  The self term -ke alpha q_j^2 / sqrt(pi) goes to E_j.
#include <cmath>
#include <complex>
#include <type_traits>
#include <vector>

#include "spme.cuh"

namespace otf {
namespace {

constexpr double kFix = 1099511627776.0;  // 2^40: fixed-point scale of the mixed form's charge mesh
// FP64 form: each mesh point is a 128-bit two's-complement integer (a low
// and a high 64-bit word) counting units of 2^-80 of a charge, so the
// quantisation (2^-81 per added value) is far below FP64 rounding and the
// range (2^47 charges) cannot be reached.
constexpr double kPi = 3.14159265358979323846;

template <typename T>
struct Rec;
template <>
struct Rec<float> {
  using type = float4;
};
template <>
struct Rec<double> {
  using type = dvec4;
};
template <typename T>
struct Cplx;
template <>
struct Cplx<float> {
  using type = cufftComplex;
};
template <>
struct Cplx<double> {
  using type = cufftDoubleComplex;
};

__device__ __forceinline__ long long to_fix(float v) { return __float2ll_rn(v * (float)kFix); }

// Adds v to mesh point idx of a mesh of K3 points: one 64-bit word per point
// (mixed form) or 128 bits per point, low words [0, K3) and high words
// [K3, 2 K3) (FP64).  The 128-bit addend is round(v 2^80) split as
// hi 2^64 + lo with lo in [0, 2^64); the carry out of the low word is the
// unsigned wrap of that add, so every order of the adds gives the same
// integer.
__device__ __forceinline__ void mesh_add(unsigned long long *Q, int64_t idx, int64_t K3, float v) {
  const long long f = to_fix(v);
  if (f != 0) atomicAdd(Q + idx, (unsigned long long)f);
}
__device__ __forceinline__ void mesh_add(unsigned long long *Q, int64_t idx, int64_t K3, double v) {
  if (v == 0.0) return;
  const double t = v * 65536.0;  // v 2^16: the high word's units (exact)
  const double fh = floor(t);
  // t - fh is exact and at most 1 - 2^-53, so its product with 2^64 is at
  // most 2^64 - 2^11 and rounds to an integer below 2^64
  const unsigned long long l = __double2ull_rn((t - fh) * 18446744073709551616.0);
  long long hi = (long long)fh;
  if (l != 0ull) {
    const unsigned long long old = atomicAdd(Q + idx, l);
    if (old + l < old) hi += 1;  // carry
  }
  if (hi != 0) atomicAdd(Q + K3 + idx, (unsigned long long)hi);
}

// Mesh coordinates of atom i: base mesh point and fraction per axis, from
// the cell index and the offset from the cell centre (FP64).  The base is
// not wrapped into [0, K) (an atom that has left its cell since the last
// sort may sit just outside the box), so that the mesh points of one cell
// row stay contiguous; mesh indices are wrapped where the mesh is read or
// written.
template <typename T>
__device__ __forceinline__ void mesh_coords(const SpmeAtoms &a, int64_t i, double kl, int K,
                                            const typename Rec<T>::type &r, int (&base)[3], T (&frac)[3]) {
  const int c = a.cpk[i];
  const int cc[3] = {c & 1023, (c >> 10) & 1023, c >> 20};
  const double off[3] = {(double)r.x, (double)r.y, (double)r.z};
  float lo[3] = {0.f, 0.f, 0.f};
  if constexpr (std::is_same<T, float>::value) {
    const float4 l4 = a.rlo[i];
    lo[0] = l4.x, lo[1] = l4.y, lo[2] = l4.z;
  }
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    double x = (cc[ax] + 0.5) * a.edge + off[ax];
    if constexpr (std::is_same<T, float>::value) x += (double)lo[ax];
    const double u = x * kl;
    const int b = (int)floor(u);
    base[ax] = b;
    frac[ax] = (T)(u - b);
  }
}

// Cardinal B-spline weights m[t] = M_N(w + t), t = 0..N-1, by the
// recursion M_p(x) = (x M_{p-1}(x) + (p - x) M_{p-1}(x - 1)) / (p - 1)
// from M_2; with derivatives, d1[t] = M_{N-1}(w+t) - M_{N-1}(w+t-1) and
// d2[t] = M_{N-2}(w+t) - 2 M_{N-2}(w+t-1) + M_{N-2}(w+t-2).
template <typename T, int N, bool DERIV>
__device__ __forceinline__ void spline(T w, T (&m)[N], T (&d1)[N], T (&d2)[N]) {
  T b[N];
  b[0] = w;
  b[1] = T(1) - w;
#pragma unroll
  for (int k = 2; k < N; ++k) b[k] = T(0);
  T o2[N], o1[N];
  if (N - 2 == 2) {
#pragma unroll
    for (int k = 0; k < N; ++k) o2[k] = b[k];
  }
#pragma unroll
  for (int p = 3; p <= N; ++p) {
    const T inv = T(1) / T(p - 1);
#pragma unroll
    for (int k = p - 1; k >= 0; --k) {
      const T prev = k > 0 ? b[k - 1] : T(0);
      b[k] = ((w + T(k)) * b[k] + (T(p) - w - T(k)) * prev) * inv;
    }
    if (p == N - 2) {
#pragma unroll
      for (int k = 0; k < N; ++k) o2[k] = b[k];
    }
    if (p == N - 1) {
#pragma unroll
      for (int k = 0; k < N; ++k) o1[k] = b[k];
    }
  }
#pragma unroll
  for (int k = 0; k < N; ++k) m[k] = b[k];
  if (DERIV) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      d1[k] = o1[k] - (k > 0 ? o1[k - 1] : T(0));
      d2[k] = o2[k] - T(2) * (k > 0 ? o2[k - 1] : T(0)) + (k > 1 ? o2[k - 2] : T(0));
    }
  }
}

__device__ __forceinline__ int wrap(int v, int K) { return ((v % K) + K) % K; }
// wrap() without the divisions for the usual case v in [-K, 2K) (mesh points
// of atoms at most a cell outside the box), with wrap() as the fallback.
__device__ __forceinline__ int wrap_near(int v, int K) {
  int w = v < 0 ? v + K : v;
  w = w >= K ? w - K : w;
  return (unsigned)w < (unsigned)K ? w : wrap(v, K);
}

constexpr int kRowThreads = 128;       // atoms per tile (one CTA)
constexpr int kTileBytes = 48 * 1024;  // shared mesh tile of the gather
constexpr int kSpreadTileBytes = 32 * 1024;  // shared mesh tile of the spread
constexpr int kChunkSlots = 8;         // CTAs per cell row (each takes every 8th chunk)
constexpr int kLoBits = 20;            // tile sums: fixed-point value = (hi << 20) + lo

template <typename T>
struct Two;
template <>
struct Two<float> {
  using type = float2;
};
template <>
struct Two<double> {
  using type = double2;
};

// The mesh points of an atom: (base - t0, base - t1, base - t2) for
// t = 0..N-1.  TILE: into a shared box of (ex, ey, ez) points whose corner
// is mesh point (ox, oy, oz) (unwrapped); otherwise into the wrapped global
// mesh.
template <typename T, int N, bool TILE>
__device__ __forceinline__ void spread_atom(const int (&base)[3], const T (&frac)[3], T q, unsigned long long *dst,
                                            int *hi, int *lo, int K, int ox, int oy, int oz, int ey, int ez) {
  const int64_t K3 = (int64_t)K * K * K;
  T wx[N], wy[N], wz[N], d1[N], d2[N];
  spline<T, N, false>(frac[0], wx, d1, d2);
  spline<T, N, false>(frac[1], wy, d1, d2);
  spline<T, N, false>(frac[2], wz, d1, d2);
  int iz[N];
#pragma unroll
  for (int t = 0; t < N; ++t) iz[t] = TILE ? base[2] - t - oz : wrap_near(base[2] - t, K);
  for (int t0 = 0; t0 < N; ++t0) {
    const int ix = TILE ? base[0] - t0 - ox : wrap_near(base[0] - t0, K);
    const T qx = q * wx[t0];
    for (int t1 = 0; t1 < N; ++t1) {
      const int iy = TILE ? base[1] - t1 - oy : wrap_near(base[1] - t1, K);
      const T qxy = qx * wy[t1];
      const int64_t row = TILE ? ((int64_t)ix * ey + iy) * ez : ((int64_t)ix * K + iy) * K;
#pragma unroll
      for (int t2 = 0; t2 < N; ++t2) {
        if (TILE) {
          // two native 32-bit shared adds: the high part (arithmetic shift)
          // and the low 20 bits; neither can overflow over one chunk
          const long long v = to_fix((float)(qxy * wz[t2]));
          atomicAdd(hi + row + iz[t2], (int)(v >> kLoBits));
          atomicAdd(lo + row + iz[t2], (int)(v & ((1ll << kLoBits) - 1)));
        } else {
          mesh_add(dst, row + iz[t2], K3, qxy * wz[t2]);
        }
      }
    }
  }
}

// The tile of one chunk of a cell row: the box of mesh points its atoms
// touch, from the block-wide extremes of their base points.
struct Tile {
  int ox, oy, oz, ex, ey, ez;
  __device__ int64_t vol() const { return (int64_t)ex * ey * ez; }
};
template <int N>
__device__ __forceinline__ Tile chunk_tile(const int (&base)[3], bool live, int *bmin, int *bmax) {
  if (threadIdx.x < 3) {
    bmin[threadIdx.x] = 0x7fffffff;
    bmax[threadIdx.x] = -0x7fffffff;
  }
  __syncthreads();
  if (live)
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      atomicMin(&bmin[ax], base[ax]);
      atomicMax(&bmax[ax], base[ax]);
    }
  __syncthreads();
  Tile t;
  t.ox = bmin[0] - (N - 1);
  t.oy = bmin[1] - (N - 1);
  t.oz = bmin[2] - (N - 1);
  t.ex = bmax[0] - bmin[0] + N;
  t.ey = bmax[1] - bmin[1] + N;
  t.ez = bmax[2] - bmin[2] + N;
  return t;
}

// Charge spreading: the atoms of a cell row in chunks of kRowThreads, one
// CTA per chunk (kChunkSlots CTAs per row).  The chunk's atoms put their bases and spline weights (q M_n in x)
// in shared memory; the chunk's tile of mesh points is then summed column
// by column (x, y fixed, z running), each column by one thread in the
// order of the atoms, so no atomic is needed inside the tile and the sums
// do not depend on scheduling; the tile's non-zero points go to the global
// mesh in 64-bit fixed point (integer atomics: order-independent).  A chunk
// whose tile does not fit (its atoms straddle the box edge) spreads atom by
// atom straight into the global mesh.
template <typename T, int N>
__global__ void __launch_bounds__(kRowThreads) k_spme_spread(SpmeAtoms a, int K, double kl, unsigned long long *Qi) {
  using R = typename Rec<T>::type;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int sb[3][kRowThreads];
  __shared__ T sw[3][N][kRowThreads];  // q M_n(x), M_n(y), M_n(z) per atom
  __shared__ int bmin[3], bmax[3];
  T *tile = reinterpret_cast<T *>(smraw);
  constexpr int64_t cap = kSpreadTileBytes / sizeof(T);
  const R *rel = static_cast<const R *>(a.rel);
  const int64_t nwork = (int64_t)a.nc * a.nc * kChunkSlots;
  for (int64_t wk = blockIdx.x; wk < nwork; wk += gridDim.x) {
    const int row = (int)(wk / kChunkSlots), slot = (int)(wk % kChunkSlots);
    const int a0 = a.cellstart[(int64_t)row * a.nc], a1 = a.cellstart[(int64_t)row * a.nc + a.nc];
    for (int c0 = a0 + slot * kRowThreads; c0 < a1; c0 += kChunkSlots * kRowThreads) {
      const int64_t i = c0 + threadIdx.x;
      const bool live = i < a1;
      const int na = min(kRowThreads, a1 - c0);
      int base[3] = {0, 0, 0};
      T frac[3] = {T(0), T(0), T(0)};
      T q = T(0);
      if (live) {
        const R r = rel[i];
        mesh_coords<T>(a, i, kl, K, r, base, frac);
        q = (T)r.w;
      }
      const Tile tl = chunk_tile<N>(base, live, bmin, bmax);
      // pad the column length to an odd number of words (no bank conflicts)
      const int ezp = tl.ez | 1;
      if ((int64_t)tl.ex * tl.ey * ezp <= cap) {
        if (live) {
          T w[3][N], d1[N], d2[N];
          spline<T, N, false>(frac[0], w[0], d1, d2);
          spline<T, N, false>(frac[1], w[1], d1, d2);
          spline<T, N, false>(frac[2], w[2], d1, d2);
#pragma unroll
          for (int t = 0; t < N; ++t) {
            sw[0][t][threadIdx.x] = q * w[0][t];
            sw[1][t][threadIdx.x] = w[1][t];
            sw[2][t][threadIdx.x] = w[2][t];
          }
#pragma unroll
          for (int ax = 0; ax < 3; ++ax) sb[ax][threadIdx.x] = base[ax];
        }
        __syncthreads();
        const int ncol = tl.ex * tl.ey;
        for (int col = threadIdx.x; col < ncol; col += kRowThreads) {
          const int lx = col / tl.ey, ly = col % tl.ey;
          T *cz = tile + (int64_t)col * ezp;
          for (int z = 0; z < tl.ez; ++z) cz[z] = T(0);
          const int gx = tl.ox + lx, gy = tl.oy + ly;
          for (int j = 0; j < na; ++j) {
            const int tx = sb[0][j] - gx, ty = sb[1][j] - gy;
            if (tx < 0 || tx >= N || ty < 0 || ty >= N) continue;
            const T c = sw[0][tx][j] * sw[1][ty][j];
            T *zz = cz + (sb[2][j] - tl.oz);
#pragma unroll
            for (int t = 0; t < N; ++t) zz[-t] += c * sw[2][t][j];
          }
        }
        __syncthreads();
        for (int col = threadIdx.x; col < ncol; col += kRowThreads) {
          const int lx = col / tl.ey, ly = col % tl.ey;
          const int64_t g0 = ((int64_t)wrap_near(tl.ox + lx, K) * K + wrap_near(tl.oy + ly, K)) * K;
          const T *cz = tile + (int64_t)col * ezp;
          for (int z = 0; z < tl.ez; ++z) mesh_add(Qi, g0 + wrap_near(tl.oz + z, K), (int64_t)K * K * K, cz[z]);
        }
      } else if (live) {
        spread_atom<T, N, false>(base, frac, q, Qi, nullptr, nullptr, K, 0, 0, 0, 0, 0);
      }
      __syncthreads();  // the tile, the atom table and the extremes are reused by the next chunk
    }
  }
}

template <typename T>
__global__ void k_spme_unfix(const unsigned long long *Qi, T *Qr, int64_t total) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (std::is_same<T, double>::value)  // hi 2^-16 + lo 2^-80
      Qr[k] = (double)(long long)Qi[total + k] * (1.0 / 65536.0) + (double)Qi[k] * 8.271806125530277e-25;
    else
      Qr[k] = (T)((double)(long long)Qi[k] * (1.0 / kFix));
  }
}

// The two convolutions on the half spectrum [K][K][K/2+1].
template <typename T>
__global__ void k_spme_conv(typename Cplx<T>::type *G1, typename Cplx<T>::type *G2, const T *bmod, int K, T invL,
                            T pa2, T cpre) {
  const int kh = K / 2 + 1;
  const int64_t total = (int64_t)K * K * kh;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int iz = (int)(e % kh);
    const int iy = (int)((e / kh) % K);
    const int ix = (int)(e / ((int64_t)kh * K));
    const T mx = (ix <= K / 2 ? ix : ix - K) * invL;
    const T my = (iy <= K / 2 ? iy : iy - K) * invL;
    const T mz = iz * invL;
    const T m2 = mx * mx + my * my + mz * mz;
    typename Cplx<T>::type g = G1[e];
    if (m2 == T(0)) {
      g.x = g.y = T(0);
      G1[e] = g;
      G2[e] = g;
      continue;
    }
    const T t = pa2 * m2;
    const T bc = bmod[ix] * bmod[iy] * bmod[iz] * exp(-t) / m2 * cpre;
    const T bh = bc * T(2) * (T(1) + t) / m2;
    typename Cplx<T>::type a = g, b = g;
    a.x *= bc;
    a.y *= bc;
    b.x *= bh;
    b.y *= bh;
    G1[e] = a;
    G2[e] = b;
  }
}

// The sums of one atom over its mesh points: energy (phi), force (first
// derivatives, phi) and the six virial sums (second derivatives, psi).
template <typename T, int N, bool TILE>
__device__ __forceinline__ void gather_atom(const int (&base)[3], const T (&frac)[3], const T *phi, const T *psi,
                                            const typename Two<T>::type *tile, int K, int ox, int oy, int oz, int ey,
                                            int ez, T (&acc)[10]) {
  T w0[N], w1[N], w2[N], d0[N], d1[N], d2[N], e0[N], e1[N], e2[N];
  spline<T, N, true>(frac[0], w0, d0, e0);
  spline<T, N, true>(frac[1], w1, d1, e1);
  spline<T, N, true>(frac[2], w2, d2, e2);
  int iz[N];
#pragma unroll
  for (int t = 0; t < N; ++t) iz[t] = TILE ? base[2] - t - oz : wrap_near(base[2] - t, K);
#pragma unroll
  for (int k = 0; k < 10; ++k) acc[k] = T(0);
  for (int t0 = 0; t0 < N; ++t0) {
    const int ix = TILE ? base[0] - t0 - ox : wrap_near(base[0] - t0, K);
#pragma unroll
    for (int t1 = 0; t1 < N; ++t1) {
      const int iy = TILE ? base[1] - t1 - oy : wrap_near(base[1] - t1, K);
      const int64_t row = TILE ? ((int64_t)ix * ey + iy) * ez : ((int64_t)ix * K + iy) * K;
      const T ww = w0[t0] * w1[t1], dw = d0[t0] * w1[t1], wd = w0[t0] * d1[t1];
      const T ew = e0[t0] * w1[t1], we = w0[t0] * e1[t1], dd = d0[t0] * d1[t1];
#pragma unroll
      for (int t2 = 0; t2 < N; ++t2) {
        T p, s;
        if (TILE) {
          const typename Two<T>::type v = tile[row + iz[t2]];
          p = v.x;
          s = v.y;
        } else {
          p = phi[row + iz[t2]];
          s = psi[row + iz[t2]];
        }
        const T pw = p * w2[t2], sw = s * w2[t2], sd = s * d2[t2];
        acc[0] += ww * pw;
        acc[1] += dw * pw;
        acc[2] += wd * pw;
        acc[3] += ww * d2[t2] * p;
        acc[4] += ew * sw;
        acc[5] += we * sw;
        acc[6] += ww * e2[t2] * s;
        acc[7] += dd * sw;
        acc[8] += dw * sd;
        acc[9] += wd * sd;
      }
    }
  }
}

// Gather, one CTA per chunk of a cell row (as the spread): the chunk's tile of (phi, psi) is
// staged in shared memory (one coalesced read per mesh point instead of one
// per atom touching it), then every atom sums over its points.
template <typename T, int N>
__global__ void __launch_bounds__(kRowThreads, 4) k_spme_gather(SpmeAtoms a, int K, double kl, const T *phi,
                                                             const T *psi, T ke, T kL, T cw, T self, T *F, T *epot,
                                                             T *W) {
  using R = typename Rec<T>::type;
  using T2 = typename Two<T>::type;
  extern __shared__ __align__(16) unsigned char smraw[];
  T2 *tile = reinterpret_cast<T2 *>(smraw);
  __shared__ int bmin[3], bmax[3];
  const R *rel = static_cast<const R *>(a.rel);
  const int64_t n = a.n;
  constexpr int64_t cap = kTileBytes / sizeof(T2);
  const int64_t nwork = (int64_t)a.nc * a.nc * kChunkSlots;
  for (int64_t wk = blockIdx.x; wk < nwork; wk += gridDim.x) {
    const int row = (int)(wk / kChunkSlots), slot = (int)(wk % kChunkSlots);
    const int a0 = a.cellstart[(int64_t)row * a.nc], a1 = a.cellstart[(int64_t)row * a.nc + a.nc];
    for (int c0 = a0 + slot * kRowThreads; c0 < a1; c0 += kChunkSlots * kRowThreads) {
      const int64_t i = c0 + threadIdx.x;
      const bool live = i < a1;
      int base[3] = {0, 0, 0};
      T frac[3] = {T(0), T(0), T(0)};
      T q = T(0);
      if (live) {
        const R r = rel[i];
        mesh_coords<T>(a, i, kl, K, r, base, frac);
        q = (T)r.w;
      }
      const Tile tl = chunk_tile<N>(base, live, bmin, bmax);
      const bool tiled = tl.vol() <= cap;
      if (tiled) {
        // element k = (lx * ey + ly) * ez + lz of the tile; consecutive threads
        // take consecutive z (coalesced), and each thread steps its (lx, ly,
        // lz) by the mixed-radix digits of the stride instead of dividing
        const int vol = (int)tl.vol();
        const int dz = kRowThreads % tl.ez, qz = kRowThreads / tl.ez, dy = qz % tl.ey, dx = qz / tl.ey;
        int lz = threadIdx.x % tl.ez, ly = (threadIdx.x / tl.ez) % tl.ey, lx = threadIdx.x / (tl.ez * tl.ey);
        for (int k = threadIdx.x; k < vol; k += kRowThreads) {
          const int64_t g =
              ((int64_t)wrap_near(tl.ox + lx, K) * K + wrap_near(tl.oy + ly, K)) * K + wrap_near(tl.oz + lz, K);
          T2 v;
          v.x = phi[g];
          v.y = psi[g];
          tile[k] = v;
          lz += dz;
          ly += dy;
          lx += dx;
          if (lz >= tl.ez) {
            lz -= tl.ez;
            ++ly;
          }
          if (ly >= tl.ey) {
            ly -= tl.ey;
            ++lx;
          }
        }
      }
      __syncthreads();
      if (live) {
        T acc[10];
        if (tiled)
          gather_atom<T, N, true>(base, frac, phi, psi, tile, K, tl.ox, tl.oy, tl.oz, tl.ey, tl.ez, acc);
        else
          gather_atom<T, N, false>(base, frac, phi, psi, tile, K, 0, 0, 0, 0, 0, acc);
        const T er = T(0.5) * ke * q * acc[0];
        epot[i] += er - self * q * q;
        const T fq = -ke * q * kL;
        F[i] += fq * acc[1];
        F[n + i] += fq * acc[2];
        F[2 * n + i] += fq * acc[3];
        const T wq = cw * q;
        W[i] += er + wq * acc[4];
        W[n + i] += er + wq * acc[5];
        W[2 * n + i] += er + wq * acc[6];
        W[3 * n + i] += wq * acc[7];
        W[4 * n + i] += wq * acc[8];
        W[5 * n + i] += wq * acc[9];
      }
      __syncthreads();
    }
  }
}

// M_n at the integers 1..n-1 (host, FP64), for the b(m) moduli.
std::vector<double> spline_at_integers(int n) {
  std::vector<double> b(n, 0.0);
  b[0] = 0.0;  // M_2 at w = 0: M_2(0) = 0, M_2(1) = 1
  b[1] = 1.0;
  for (int p = 3; p <= n; ++p)
    for (int k = p - 1; k >= 0; --k) b[k] = ((double)k * b[k] + (double)(p - k) * (k > 0 ? b[k - 1] : 0.0)) / (p - 1);
  return b;  // b[k] = M_n(k)
}

int cufft_ok(cufftResult r, const char *what) {
  if (r == CUFFT_SUCCESS) return MD_OK;
  set_error("%s failed (cuFFT error %d)", what, (int)r);
  return MD_ECUDA;
}

int grid_of(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 16); }

}  // namespace

int Spme::create(const SpmeParams &p, bool fp64, cudaStream_t st) {
  p_ = p;
  fp64_ = fp64;
  const int K = p.K;
  const int64_t K3 = (int64_t)K * K * K, KH = (int64_t)K * K * (K / 2 + 1);
  const size_t ts = fp64 ? sizeof(double) : sizeof(float);
  // |b(m)|^2 = 1 / |sum_{k=0}^{n-2} M_n(k+1) exp(2 pi i m k / K)|^2
  const std::vector<double> Mk = spline_at_integers(p.order);
  std::vector<double> bm(K);
  for (int m = 0; m < K; ++m) {
    std::complex<double> s(0.0, 0.0);
    for (int k = 0; k <= p.order - 2; ++k) s += Mk[k + 1] * std::polar(1.0, 2.0 * kPi * m * k / K);
    bm[m] = 1.0 / std::norm(s);
  }
  OTF_CUDA(cudaMalloc(&Qi_, sizeof(unsigned long long) * K3 * (fp64 ? 2 : 1)));  // 128-bit points in FP64
  OTF_CUDA(cudaMalloc(&Qr_, ts * K3));
  OTF_CUDA(cudaMalloc(&phi_, ts * K3));
  OTF_CUDA(cudaMalloc(&psi_, ts * K3));
  OTF_CUDA(cudaMalloc(&G1_, 2 * ts * KH));
  OTF_CUDA(cudaMalloc(&G2_, 2 * ts * KH));
  OTF_CUDA(cudaMalloc(&bmod_, ts * K));
  if (fp64) {
    OTF_CUDA(cudaMemcpy(bmod_, bm.data(), sizeof(double) * K, cudaMemcpyHostToDevice));
  } else {
    std::vector<float> bf(bm.begin(), bm.end());
    OTF_CUDA(cudaMemcpy(bmod_, bf.data(), sizeof(float) * K, cudaMemcpyHostToDevice));
  }
  int rc = cufft_ok(cufftPlan3d(&fwd_, K, K, K, fp64 ? CUFFT_D2Z : CUFFT_R2C), "cufftPlan3d (forward)");
  if (!rc) rc = cufft_ok(cufftPlan3d(&inv_, K, K, K, fp64 ? CUFFT_Z2D : CUFFT_C2R), "cufftPlan3d (inverse)");
  if (rc) return rc;
  plans_ = true;
  rc = cufft_ok(cufftSetStream(fwd_, st), "cufftSetStream");
  if (!rc) rc = cufft_ok(cufftSetStream(inv_, st), "cufftSetStream");
  return rc;
}

void Spme::destroy() {
  if (plans_) {
    cufftDestroy(fwd_);
    cufftDestroy(inv_);
    plans_ = false;
  }
  for (void *q : {(void *)Qi_, Qr_, phi_, psi_, G1_, G2_, bmod_})
    if (q) cudaFree(q);
  Qi_ = nullptr;
  Qr_ = phi_ = psi_ = G1_ = G2_ = bmod_ = nullptr;
}

template <typename T>
int Spme::run_t(const SpmeAtoms &a, T *F, T *epot, T *W, cudaStream_t st) {
  const int K = p_.K;
  const int64_t K3 = (int64_t)K * K * K;
  const double kl = K / p_.L;
  // the FFTs follow the caller's stream (a graph may be capturing it)
  int rs = cufft_ok(cufftSetStream(fwd_, st), "cufftSetStream");
  if (!rs) rs = cufft_ok(cufftSetStream(inv_, st), "cufftSetStream");
  if (rs) return rs;
  OTF_CUDA(cudaMemsetAsync(Qi_, 0, sizeof(unsigned long long) * K3 * (fp64_ ? 2 : 1), st));
  if (!a.cellstart || a.nc < 1) {
    set_error("spme: the cell list is missing");
    return MD_EINVAL;
  }
  const int rows = (int)std::min<int64_t>((int64_t)a.nc * a.nc * kChunkSlots, 152 * 32);
  if (!attr_) {
    for (const void *f : {(const void *)k_spme_spread<T, 4>, (const void *)k_spme_spread<T, 6>,
                          (const void *)k_spme_spread<T, 8>})
      OTF_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kSpreadTileBytes));
    for (const void *f : {(const void *)k_spme_gather<T, 4>, (const void *)k_spme_gather<T, 6>,
                          (const void *)k_spme_gather<T, 8>})
      OTF_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileBytes));
    attr_ = true;
  }
  switch (p_.order) {
    case 4:
      k_spme_spread<T, 4><<<rows, kRowThreads, kSpreadTileBytes, st>>>(a, K, kl, Qi_);
      break;
    case 6:
      k_spme_spread<T, 6><<<rows, kRowThreads, kSpreadTileBytes, st>>>(a, K, kl, Qi_);
      break;
    default:
      k_spme_spread<T, 8><<<rows, kRowThreads, kSpreadTileBytes, st>>>(a, K, kl, Qi_);
  }
  k_spme_unfix<T><<<grid_of(K3), 256, 0, st>>>(Qi_, static_cast<T *>(Qr_), K3);
  OTF_LAUNCH_CHECK();
  using C = typename Cplx<T>::type;
  int rc;
  if constexpr (std::is_same<T, double>::value)
    rc = cufft_ok(cufftExecD2Z(fwd_, static_cast<double *>(Qr_), static_cast<C *>(G1_)), "cufftExecD2Z");
  else
    rc = cufft_ok(cufftExecR2C(fwd_, static_cast<float *>(Qr_), static_cast<C *>(G1_)), "cufftExecR2C");
  if (rc) return rc;
  const double V = p_.L * p_.L * p_.L;
  k_spme_conv<T><<<grid_of((int64_t)K * K * (K / 2 + 1)), 256, 0, st>>>(
      static_cast<C *>(G1_), static_cast<C *>(G2_), static_cast<const T *>(bmod_), K, (T)(1.0 / p_.L),
      (T)(kPi * kPi / (p_.alpha * p_.alpha)), (T)(1.0 / (kPi * V)));
  OTF_LAUNCH_CHECK();
  if constexpr (std::is_same<T, double>::value) {
    rc = cufft_ok(cufftExecZ2D(inv_, static_cast<C *>(G1_), static_cast<double *>(phi_)), "cufftExecZ2D");
    if (!rc) rc = cufft_ok(cufftExecZ2D(inv_, static_cast<C *>(G2_), static_cast<double *>(psi_)), "cufftExecZ2D");
  } else {
    rc = cufft_ok(cufftExecC2R(inv_, static_cast<C *>(G1_), static_cast<float *>(phi_)), "cufftExecC2R");
    if (!rc) rc = cufft_ok(cufftExecC2R(inv_, static_cast<C *>(G2_), static_cast<float *>(psi_)), "cufftExecC2R");
  }
  if (rc) return rc;
  const T ke = (T)p_.ke, kL = (T)kl, cw = (T)(p_.ke * kl * kl / (8.0 * kPi * kPi)),
          self = (T)(p_.ke * p_.alpha / std::sqrt(kPi));
  const T *phi = static_cast<const T *>(phi_), *psi = static_cast<const T *>(psi_);
  switch (p_.order) {
    case 4:
      k_spme_gather<T, 4><<<rows, kRowThreads, kTileBytes, st>>>(a, K, kl, phi, psi, ke, kL, cw, self, F, epot, W);
      break;
    case 6:
      k_spme_gather<T, 6><<<rows, kRowThreads, kTileBytes, st>>>(a, K, kl, phi, psi, ke, kL, cw, self, F, epot, W);
      break;
    default:
      k_spme_gather<T, 8><<<rows, kRowThreads, kTileBytes, st>>>(a, K, kl, phi, psi, ke, kL, cw, self, F, epot, W);
  }
  OTF_LAUNCH_CHECK();
  return MD_OK;
}

int Spme::run(const SpmeAtoms &a, void *F, void *epot, void *W, cudaStream_t st) {
  if (fp64_)
    return run_t<double>(a, static_cast<double *>(F), static_cast<double *>(epot), static_cast<double *>(W), st);
  return run_t<float>(a, static_cast<float *>(F), static_cast<float *>(epot), static_cast<float *>(W), st);
}

}  // namespace otf
