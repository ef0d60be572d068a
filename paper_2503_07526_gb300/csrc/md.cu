// Lennard-Jones MD step with on-the-fly stress, heat flux and correlators
// (arXiv 2503.07526: Sec. 1 linked cells and velocity Verlet; Sec. 2.3
// Eq. (stress) and the heat-flux definition; Sec. 2.2 correlators).
//
// GB300 design.  Atoms live in a cell-sorted structure of arrays that is
// rebuilt by a counting sort when any atom has moved half the skin.  Each
// atom carries its coordinates relative to the centre of the cell it was
// sorted into (|rel| <= edge/2) in the arithmetic type of the pair path, so
// the FP32 form never subtracts two large absolute coordinates.
//
// State.  The FP64 form keeps absolute FP64 positions and velocities.  The
// mixed form keeps each position as a cell index plus a double-float offset
// from that cell's centre (the high words are the FP32 coordinates the pair
// kernel reads) and each velocity as a double-float: about 48 significant
// bits, integrated with FP32 error-free transformations, because GB300's
// FP64 pipe runs at a small fraction of its FP32 rate.  Moving an atom to
// another cell shifts its offset by whole cell edges; crossing the periodic
// boundary only changes the cell index.
//
// Neighbour lists.  MD_PAIR_VERLET stores them per chunk of up to 32
// consecutive atoms: a block of max_neighbors rows of 32 words (atom index
// and image code), so the list build writes rows that stay together in L2
// and the pair kernel reads them coalesced.  MD_PAIR_TILES (the mixed
// Lennard-Jones form) cuts the cells into tiles; a tile's CTA stages the
// tile and its one-cell shell in shared memory in the tile's own frame, and
// the lists hold 16-bit byte offsets into that window (see the tile-window
// section below).
//
// Replicas.  One handle can hold many independent systems ("replicas", of
// uneven sizes, densities and temperatures).  Their atoms, cells and
// reduction CTAs are laid end to end and every kernel covers all of them at
// once, looking up a replica's box, cell grid and offsets in a small
// descriptor table; a single system is one replica.
//
// A step is a fixed sequence of kernels (no host decision inside it), so it
// is captured once as a CUDA graph and replayed; the rebuild kernels read a
// device flag and return at once when no rebuild is due.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include <cuda_fp16.h>

#include "corr.cuh"
#include "spme.cuh"

namespace otf {
namespace {

constexpr int kThreads = 256;
constexpr int kGraphSteps = 8;  // steps per replayed graph (velocity pushes overlap the next step)
constexpr int kDefaultBuildKind = 0;  // list build without autotuning: 0 j-parallel, 1 i-parallel, 2 staged
constexpr int kPairThreads = 128;     // default CTA of the pair kernel (the autotuner may pick 64 or 256)
constexpr int kMaxPairThreads = 256;
constexpr int kCellWarps = 4;  // warps (cells) per CTA in the link-cell kernels
constexpr int kNRed = 14;      // K, U, V*sigma[6], V*q[3], V*j[3]
constexpr int kNBanks = 4;     // stress, heat flux, velocity, mass flux
constexpr int kMaxRedBlocks = 152 * 64;  // reduction CTAs per replica at most
// atoms per reduction CTA in the mixed form (14 per thread): at 2,048,000
// atoms its 572 CTAs fill 94 % of the 608 that fit the GPU at once (four per
// SM) where 4,096 atoms per CTA left 500 (82 %, the SMs holding four CTAs
// setting the time): 0.1146 against 0.1190 ms per step, and 3,840 atoms
// 0.1169; smaller CTAs lose more to the per-CTA merge and the last CTA's pass
// (0.123 / 0.134 / 0.160 ms for 2,048 / 1,024 / 512 atoms)
constexpr int kRedAtomsMixed = 3584;
constexpr double kRClose = 1.03;  // close-pair radius of the mixed form, in sigma

// Step counters shared by all replicas.
struct StepDev {
  int64_t step;       // steps completed
  int64_t corr_base;  // step at the last correlator reset
  int64_t rebuilds;   // neighbour-list / cell rebuilds since md_init
  unsigned reps_done; // replicas whose reduction finished in this launch
  unsigned vacf_ctas; // CTAs of a blocked velocity push that have finished (returns to 0)
  int64_t vacf_done;  // velocity-correlator pushes applied (the rest wait in their input slots)
};

// Observables of one replica.
struct ObsDev {
  int64_t Tn;
  double U, K, T;
  double sigma[6];
  double q[3];
  double Tsum;
  double j[3];  // partial momentum density of the flux species
};

// Constants of one replica.  Its atoms occupy [atom0, atom1) of the
// cell-sorted order (the counting sort never moves an atom across replicas,
// since a replica's cells are contiguous), its cells [cell0, cell0 + nc^3),
// its reduction CTAs [block0, block0 + nblk).
struct Rep {
  int64_t atom0, atom1, cell0, block0;
  int nc, nblk;
  double L, edge;
  float edge_h, edge_l;  // double-float edge (mixed form)
};

// One tile of the MD_PAIR_TILES path: cells [x0, x0 + bx) x [y0, y0 + by) x
// [z0, z0 + bz) of replica rep (a tile never wraps around the box).
struct Tile {
  int rep;
  unsigned short x0, y0, z0;
  unsigned char bx, by, bz, pad;
};

struct Sys {
  int64_t n, ncell, maxchunks;  // totals over all replicas
  int nrep, ntypes, maxnb, always_rebuild, vacf_u;
  int vacf_slots;  // velocity input slots: kPushBlock (blocked pushes), 1 (one push per step) or 0 (off)
  double dt, lim2;
  double invm[8], mass[8];
  double charge[8];            // per type (MD_POT_BUCK_EWALD); the pair records carry it in w
  int flux_species;            // type whose partial momentum density is observed
  int unit_mass;               // every type's mass is exactly 1 (m v needs no product)
  float hdtm_h[8], hdtm_l[8];  // mixed form: dt / (2 m) per type, double-float
  float mass_h[8], mass_l[8];  // mixed form: m per type, double-float
  float dt_h, dt_l;
  const Rep *rep;            // [nrep]
  const int *rep_of_atom;    // [n] (sorted order = input order of replicas)
  const int *rep_of_cell;    // [ncell]
  const int *rep_of_block;   // [reduction CTAs]
  const double *lam;         // [nrep] velocity scale factors (md_scale_velocities)
  // cell-sorted state
  double *r, *v;             // FP64 form: absolute positions, velocities [3][n]
  float4 *rlo;               // mixed form: offset low words (x, y, z, 0) [n]
  float *vh, *vl;            // mixed form: velocity words [3][n]
  void *F, *epot, *W;        // [3][n], [n], [6][n] in the pair type
  void *rel, *relb;          // Vec4 of the pair type: current / at last rebuild
  void *vbuf;                // [vacf_slots][3][n] velocities in atom-id order, one slot per waiting
                             // velocity-correlator push ((push - 1) mod vacf_slots)
  int *id, *type, *cpk;      // atom id, type, packed cell coordinates
  // rebuild scratch (24 bytes per atom each)
  double *rB, *vB;
  int *idB, *typeB, *cellB, *slot, *perm, *cellcount, *cellstart;
  uint32_t *nbr;             // [n/32 chunks][maxnb][32]: j << 6 | image code
  int *nnb;                  // list length per atom (MD_PAIR_TILES: far | close << 16)
  // MD_PAIR_TILES
  const Tile *tiles;         // [ntiles]
  int ntiles, wcap;          // tiles; window slots per tile (slot 0: the far-away dummy)
  uint4 *tnb;                // [maxnb / 8][n]: far entries, eight 16-bit window byte offsets per block
  uint4 *tcl;                // [kMaxCloseT / 8][n]: close entries, the same way
  struct TileWin *trec;      // [ntiles]: window layout of each tile at the last list build
  unsigned char *tcell;      // [ntiles][wcap + kWinPad]: window cell of each slot, the same
  // reductions and flags
  double *partials;          // [reduction CTAs][kNRed]
  unsigned *counter;         // [nrep] finished CTAs per replica
  ObsDev *obs;               // [nrep]
  StepDev *st;
  int *rebuild;              // [1 + nrep]: any replica, then each replica
  unsigned *err;
};

template <typename TF>
struct LJ {
  TF c12, c6, f12, f6;  // 4 eps sig^12, 4 eps sig^6, 12 c12, 6 c6
  TF rc2, ushift, rlist2;
  TF rclose2;           // mixed form: pairs closer than r_close get the rounded-once displacement
  TF rcb2;              // MD_PAIR_TILES: (r_close + skin)^2, the list build's close segment
  // MD_POT_BUCK_EWALD: A exp(-r/rho) - C/r^6 + ke qq erfc(alpha r)/r
  TF A, inv_rho, C6, alpha, c2, ke;  // c2 = 2 alpha / sqrt(pi)
};
constexpr int kPotLJ = 0, kPotBuck = 1;

__device__ __forceinline__ int pack_cell(int x, int y, int z) { return x | (y << 10) | (z << 20); }
__device__ __forceinline__ void unpack_cell(int c, int &x, int &y, int &z) {
  x = c & 1023;
  y = (c >> 10) & 1023;
  z = c >> 20;
}
__device__ __forceinline__ int type_of(const Sys &d, int64_t i) { return min(max(d.type[i], 0), 7); }
__device__ __forceinline__ const Rep &rep_of(const Sys &d, int64_t i) { return d.rep[d.rep_of_atom[i]]; }
// Rebuild flags: a replica is re-sorted and gets new lists only when one of
// its own atoms has moved half the skin, so each replica follows exactly the
// schedule it would follow alone.
__device__ __forceinline__ bool any_rebuild(const Sys &d) { return d.rebuild[0] != 0; }
__device__ __forceinline__ bool rebuilds(const Sys &d, int r) { return d.rebuild[1 + r] != 0; }
__device__ __forceinline__ void request_rebuild(const Sys &d, int r) {
  d.rebuild[1 + r] = 1;
  d.rebuild[0] = 1;
}

// ------------------------------------------------------------ integrate

// FP64 form: first half kick and drift (velocity Verlet), new
// cell-relative coordinates, and the skin test that decides the next
// rebuild.
// Link-cell mode (or no skin): every replica is re-sorted every step.
__device__ __forceinline__ void request_all(const Sys &d) {
  if (d.always_rebuild && blockIdx.x == 0)
    for (int k = threadIdx.x; k <= d.nrep; k += blockDim.x) d.rebuild[k] = 1;
}

__global__ void __launch_bounds__(kThreads) k_kick_drift64(Sys d, double hdt) {
  request_all(d);
  const double *F = static_cast<const double *>(d.F);
  dvec4 *rel = static_cast<dvec4 *>(d.rel);
  const dvec4 *relb = static_cast<const dvec4 *>(d.relb);
  bool bad = false;
  const int64_t n = d.n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double h = hdt * d.invm[type_of(d, i)];
    // every load first (the stores below could alias them for the compiler)
    double fa[3], va0[3], ra[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      fa[a] = F[a * n + i];
      va0[a] = d.v[a * n + i];
      ra[a] = d.r[a * n + i];
    }
    const double qw = rel[i].w;
    const dvec4 b = Vec4<double>::load(relb + i);
    double x[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double va = fma(h, fa[a], va0[a]);
      d.v[a * n + i] = va;
      x[a] = fma(d.dt, va, ra[a]);
      d.r[a * n + i] = x[a];
    }
    int cx, cy, cz;
    unpack_cell(d.cpk[i], cx, cy, cz);
    const double edge = rep_of(d, i).edge;
    const double px = fma(-(cx + 0.5), edge, x[0]);
    const double py = fma(-(cy + 0.5), edge, x[1]);
    const double pz = fma(-(cz + 0.5), edge, x[2]);
    Vec4<double>::store(rel + i, px, py, pz, qw);
    const double dx = px - b.x, dy = py - b.y, dz = pz - b.z;
    if ((dx * dx + dy * dy + dz * dz) > d.lim2) request_rebuild(d, d.rep_of_atom[i]);
    bad |= !(isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]));
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(d.err, ERR_NONFINITE);
}

// Mixed form: the same half kick and drift in double-float arithmetic on
// the velocity and on the offset from the cell centre (no FP64 instruction
// per atom).  The offset's high words are the FP32 coordinates of the pair
// kernel.
__global__ void __launch_bounds__(kThreads) k_kick_drift_df(Sys d) {
  request_all(d);
  const float *F = static_cast<const float *>(d.F);
  float4 *rel = static_cast<float4 *>(d.rel);
  const float4 *relb = static_cast<const float4 *>(d.relb);
  const dfloat dt{d.dt_h, d.dt_l};
  const float lim2 = (float)d.lim2;
  bool bad = false;
  const int64_t n = d.n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int t = type_of(d, i);
    // every load first (the stores below could alias them for the compiler)
    const float4 o = rel[i];
    const float4 b = relb[i];
    const float4 lo = d.rlo[i];
    const float ol[3] = {lo.x, lo.y, lo.z};
    float fa[3], vh[3], vl[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      fa[a] = F[a * n + i];
      vh[a] = d.vh[a * n + i];
      vl[a] = d.vl[a * n + i];
    }
    const dfloat h{d.hdtm_h[t], d.hdtm_l[t]};
    float oh[3] = {o.x, o.y, o.z}, nl[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      dfloat v{vh[a], vl[a]};
      v = df_add(v, df_mul_f(h, fa[a]));
      d.vh[a * n + i] = v.h;
      d.vl[a * n + i] = v.l;
      dfloat x{oh[a], ol[a]};
      x = df_add(x, df_mul(dt, v));
      oh[a] = x.h;
      nl[a] = x.l;
    }
    rel[i] = make_float4(oh[0], oh[1], oh[2], o.w);
    d.rlo[i] = make_float4(nl[0], nl[1], nl[2], 0.f);
    const float dx = oh[0] - b.x, dy = oh[1] - b.y, dz = oh[2] - b.z;
    if ((dx * dx + dy * dy + dz * dz) > lim2) request_rebuild(d, d.rep_of_atom[i]);
    bad |= !(isfinite(oh[0]) && isfinite(oh[1]) && isfinite(oh[2]));
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(d.err, ERR_NONFINITE);
}

// ---------------------------------------------------------------- sort

__global__ void k_rb_zero(Sys d) {
  if (!any_rebuild(d)) return;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < d.ncell;
       c += (int64_t)gridDim.x * blockDim.x)
    if (rebuilds(d, d.rep_of_cell[c])) d.cellcount[c] = 0;
}

// Takes a provisional slot in cell c for atom i: lanes binning into the
// same cell share one atomic (consecutive atoms are mostly in one cell).
__device__ __forceinline__ void bin_atom(const Sys &d, int64_t i, int c) {
  d.cellB[i] = c;
  const unsigned grp = __match_any_sync(__activemask(), c);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(grp) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(&d.cellcount[c], __popc(grp));
  base = __shfl_sync(grp, base, leader);
  d.slot[i] = base + __popc(grp & ((1u << lane) - 1u));
}

// FP64 form: wraps positions into the box, bins every atom into its cell
// and copies the state aside for the gather.
__global__ void __launch_bounds__(kThreads) k_rb_assign64(Sys d) {
  if (!any_rebuild(d)) return;
  const int64_t n = d.n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!rebuilds(d, d.rep_of_atom[i])) continue;
    const Rep &R = rep_of(d, i);
    const int nc = R.nc;
    int ci[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double x = d.r[a * n + i];
      x -= R.L * floor(x / R.L);
      if (x >= R.L) x -= R.L;
      if (x < 0.0) x = 0.0;
      const int c = (int)(x / R.edge);
      ci[a] = c < nc ? c : nc - 1;
      d.rB[a * n + i] = x;
      d.vB[a * n + i] = d.v[a * n + i];
    }
    const int t = d.type[i];
    if (t < 0 || t >= d.ntypes) atomicOr(d.err, ERR_BAD_TYPE);
    d.idB[i] = d.id[i];
    d.typeB[i] = t;
    bin_atom(d, i, (int)R.cell0 + (ci[2] * nc + ci[1]) * nc + ci[0]);
  }
}

// Mixed form: the new cell is the old one moved by the nearest whole number
// of cell edges along each axis (periodic), and the offset loses the same
// multiple of the edge, in double-float.  Scratch layout: rB = offset high
// then low words, vB = velocity high then low words (float [3][n] each).
__global__ void __launch_bounds__(kThreads) k_rb_assign_df(Sys d) {
  if (!any_rebuild(d)) return;
  const int64_t n = d.n;
  const float4 *rel = static_cast<const float4 *>(d.rel);
  float *oB = reinterpret_cast<float *>(d.rB);
  float *wB = reinterpret_cast<float *>(d.vB);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!rebuilds(d, d.rep_of_atom[i])) continue;
    const Rep &R = rep_of(d, i);
    const int nc = R.nc;
    const dfloat edge{R.edge_h, R.edge_l};
    const float4 o = rel[i];
    const float4 lo = d.rlo[i];
    const float oh[3] = {o.x, o.y, o.z}, ol[3] = {lo.x, lo.y, lo.z};
    int cc[3];
    unpack_cell(d.cpk[i], cc[0], cc[1], cc[2]);
    int ci[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      dfloat x{oh[a], ol[a]};
      int k = (int)rintf(x.h / R.edge_h);  // NaN converts to 0
      k = max(-nc, min(nc, k));
      if (k != 0) x = df_add(x, df_mul_f(edge, (float)(-k)));
      int c = (cc[a] + k) % nc;
      if (c < 0) c += nc;
      ci[a] = c;
      oB[a * n + i] = x.h;
      oB[3 * n + a * n + i] = x.l;
      wB[a * n + i] = d.vh[a * n + i];
      wB[3 * n + a * n + i] = d.vl[a * n + i];
    }
    const int t = d.type[i];
    if (t < 0 || t >= d.ntypes) atomicOr(d.err, ERR_BAD_TYPE);
    d.idB[i] = d.id[i];
    d.typeB[i] = t;
    bin_atom(d, i, (int)R.cell0 + (ci[2] * nc + ci[1]) * nc + ci[0]);
  }
}

// Exclusive scan of the cell counts (one CTA of 1024 threads).  Warp w owns
// a contiguous segment and reads it in coalesced rows of 32: pass 1 sums the
// segments, warp 0 scans the 32 sums, pass 2 scans each row with shuffles
// and a running carry.
__global__ void __launch_bounds__(1024) k_rb_scan(Sys d) {
  if (!any_rebuild(d)) return;
  __shared__ int wsum[32];
  const int64_t nc3 = d.ncell;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t seg = (nc3 + 31) / 32;
  const int64_t c0 = warp * seg, c1 = min(nc3, c0 + seg);
  int part = 0;
  for (int64_t c = c0 + lane; c < c1; c += 32) part += d.cellcount[c];
  part = warp_sum(part);
  if (lane == 0) wsum[warp] = part;
  __syncthreads();
  if (warp == 0) {
    const int v = wsum[lane];
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    wsum[lane] = incl - v;  // exclusive offset of each segment
  }
  __syncthreads();
  int carry = wsum[warp];
  for (int64_t b = c0; b < c1; b += 32) {
    const int64_t c = b + lane;
    const int v = c < c1 ? d.cellcount[c] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (c < c1) d.cellstart[c] = carry + incl - v;
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (threadIdx.x == 0) {
    d.cellstart[nc3] = (int)d.n;
    d.st->rebuilds += 1;
  }
}

__global__ void __launch_bounds__(kThreads) k_rb_place(Sys d) {
  if (!any_rebuild(d)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (rebuilds(d, d.rep_of_atom[i])) d.perm[d.cellstart[d.cellB[i]] + d.slot[i]] = (int)i;
}

// Sort key of atom a (unsorted scratch index) inside its cell: the octant
// of the cell it sits in (x fastest), then its id.  Atoms of one octant are
// close, so consecutive atoms -- the lanes of a pair-kernel warp -- have
// nearly the same neighbours and gather nearby coordinates at the same list
// position.  The order is a pure function of positions and ids
// (deterministic whatever order the atomics gave).
template <typename TF>
__device__ __forceinline__ int cell_key(const Sys &d, int a, int cx, int cy, int cz, double edge) {
  int oct;
  if constexpr (std::is_same<TF, double>::value) {
    const int64_t n = d.n;
    oct = (d.rB[a] >= (cx + 0.5) * edge) | ((d.rB[n + a] >= (cy + 0.5) * edge) << 1) |
          ((d.rB[2 * n + a] >= (cz + 0.5) * edge) << 2);
  } else {
    const float *oB = reinterpret_cast<const float *>(d.rB);  // offsets from the cell centre
    const int64_t n = d.n;
    oct = (oB[a] >= 0.f) | ((oB[n + a] >= 0.f) << 1) | ((oB[2 * n + a] >= 0.f) << 2);
  }
  return (oct << 27) | d.idB[a];
}

// One warp per cell: orders the cell's atoms by (octant, id) and gathers
// them into place with their cell-relative coordinates.
template <typename TF>
__global__ void __launch_bounds__(kCellWarps * 32) k_rb_rank(Sys d) {
  if (!any_rebuild(d)) return;
  const int lane = threadIdx.x & 31;
  const int64_t n = d.n;
  const int64_t wglobal = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = wglobal; c < d.ncell; c += nwarps) {
    if (!rebuilds(d, d.rep_of_cell[c])) continue;
    const int s0 = d.cellstart[c], cnt = d.cellstart[c + 1] - s0;
    const Rep &R = d.rep[d.rep_of_cell[c]];
    const int64_t lc = c - R.cell0;
    const int cx = (int)(lc % R.nc), cy = (int)((lc / R.nc) % R.nc), cz = (int)(lc / ((int64_t)R.nc * R.nc));
    for (int e0 = 0; e0 < cnt; e0 += 32) {
      const int e = e0 + lane;
      const int a = e < cnt ? d.perm[s0 + e] : 0;
      const int key = e < cnt ? cell_key<TF>(d, a, cx, cy, cz, R.edge) : 0x7fffffff;
      int rank = 0;
      for (int f0 = 0; f0 < cnt; f0 += 32) {
        const int other = (f0 + lane < cnt) ? cell_key<TF>(d, d.perm[s0 + f0 + lane], cx, cy, cz, R.edge) : 0x7fffffff;
        for (int f = 0; f < 32; ++f) rank += (__shfl_sync(0xffffffffu, other, f) < key);
      }
      if (e < cnt) {
        const int dst = s0 + rank;
        d.id[dst] = key & 0x07ffffff;
        d.type[dst] = d.typeB[a];
        d.cpk[dst] = pack_cell(cx, cy, cz);
        if constexpr (std::is_same<TF, double>::value) {
          double x[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            x[q] = d.rB[q * n + a];
            d.r[q * n + dst] = x[q];
            d.v[q * n + dst] = d.vB[q * n + a];
          }
          const double px = fma(-(cx + 0.5), R.edge, x[0]);
          const double py = fma(-(cy + 0.5), R.edge, x[1]);
          const double pz = fma(-(cz + 0.5), R.edge, x[2]);
          const double qc = d.charge[min(max(d.typeB[a], 0), 7)];
          Vec4<double>::store(static_cast<dvec4 *>(d.rel) + dst, px, py, pz, qc);
          Vec4<double>::store(static_cast<dvec4 *>(d.relb) + dst, px, py, pz, qc);
        } else {
          const float *oB = reinterpret_cast<const float *>(d.rB);
          const float *wB = reinterpret_cast<const float *>(d.vB);
          float oh[3], ol[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            oh[q] = oB[q * n + a];
            ol[q] = oB[3 * n + q * n + a];
            d.vh[q * n + dst] = wB[q * n + a];
            d.vl[q * n + dst] = wB[3 * n + q * n + a];
          }
          d.rlo[dst] = make_float4(ol[0], ol[1], ol[2], 0.f);
          const float4 o = make_float4(oh[0], oh[1], oh[2], (float)d.charge[min(max(d.typeB[a], 0), 7)]);
          static_cast<float4 *>(d.rel)[dst] = o;
          static_cast<float4 *>(d.relb)[dst] = o;
        }
      }
    }
  }
}

// ---------------------------------------------------------------- pairs

// Neighbour-list entries: j << 6 | (oz + 1) << 4 | (oy + 1) << 2 | (ox + 1).
// (ox, oy, oz) in {-1, 0, 1}^3 is the cell of j relative to the cell of i,
// so j's offset from its own cell centre moves into i's frame by (ox, oy, oz)
// cell edges (the periodic image is implied).  26 bits of atom index.
constexpr int kEntShift = 6;
__device__ __forceinline__ uint32_t list_entry(int j, int ox, int oy, int oz) {
  return ((uint32_t)j << kEntShift) | (uint32_t)((ox + 1) | ((oy + 1) << 2) | ((oz + 1) << 4));
}
__device__ __forceinline__ int entry_atom(uint32_t e) { return (int)(e >> kEntShift); }
// The image offset as exact floats -1, 0, 1 without an integer conversion:
// OR-ing a small integer k into the mantissa of 1.5 * 2^23 gives exactly
// 1.5 * 2^23 + k, from which the constant comes off exactly.
__device__ __forceinline__ void entry_image_f(uint32_t e, float &ox, float &oy, float &oz) {
  ox = __uint_as_float(0x4B400000u | (e & 3u)) - 12582913.0f;
  oy = __uint_as_float(0x4B400000u | ((e >> 2) & 3u)) - 12582913.0f;
  oz = __uint_as_float(0x4B400000u | ((e >> 4) & 3u)) - 12582913.0f;
}
__device__ __forceinline__ void entry_image(uint32_t e, int &ox, int &oy, int &oz) {
  ox = (int)(e & 3u) - 1;
  oy = (int)((e >> 2) & 3u) - 1;
  oz = (int)((e >> 4) & 3u) - 1;
}

// Final list length of a build, clamped to the capacity (an overflow is
// reported through the error word).
__device__ __forceinline__ int list_count(const Sys &d, int cnt) {
  if (cnt > d.maxnb) atomicOr(d.err, ERR_NBR_OVERFLOW);
  return min(cnt, d.maxnb);
}

// Pair terms at squared distance r2 < rc2 (Sec. 2.3's pair potential):
// returns fs = -U'(r)/r, so that the force on i is fs d with d = r_i - r_j,
// and sets u = U(r).  Lennard-Jones, energy-shifted: U = c12 / r^12 -
// c6 / r^6 - U(rc), fs = (f12 / r^12 - f6 / r^6) / r^2 with c12 = 4 eps sig^12,
// c6 = 4 eps sig^6, f12 = 12 c12, f6 = 6 c6.  qq is the product of the two
// charges (the Buckingham + real-space Ewald form).
template <typename TF, int POT>
__device__ __forceinline__ TF pair_terms(const LJ<TF> &lj, TF r2, TF qq, TF &u) {
  if constexpr (POT == kPotLJ) {
    const TF ir2 = pair_rcp(r2);
    const TF ir6 = ir2 * ir2 * ir2;
    u = ir6 * (lj.c12 * ir6 - lj.c6) - lj.ushift;
    return ir2 * ir6 * (lj.f12 * ir6 - lj.f6);
  } else {
    // Buckingham plus the real-space Ewald term (arXiv 2503.07526 Sec. 5.3;
    // erfc screening of Essmann et al. 1995)
    const TF r = sqrt(r2);
    const TF ir = TF(1) / r;
    const TF ir2 = ir * ir;
    const TF ir6 = ir2 * ir2 * ir2;
    const TF ex = lj.A * exp(-r * lj.inv_rho);
    const TF ar = lj.alpha * r;
    const TF ec = erfc(ar);
    const TF qk = lj.ke * qq;
    u = ex - lj.C6 * ir6 + qk * ec * ir;
    const TF mdu = ex * lj.inv_rho - TF(6) * lj.C6 * ir6 * ir + qk * (ec * ir2 + lj.c2 * exp(-ar * ar) * ir);
    return mdu * ir;
  }
}

// f += fs d, e += u, w += d (x) (fs d) (the 1/2 of the per-particle split is
// applied once at the end).
template <typename TF>
__device__ __forceinline__ void pair_add(TF dx, TF dy, TF dz, TF u, TF fs, TF f[3], TF &e, TF w[6]) {
  const TF fx = fs * dx, fy = fs * dy, fz = fs * dz;
  f[0] += fx;
  f[1] += fy;
  f[2] += fz;
  e += u;
  w[0] += dx * fx;
  w[1] += dy * fy;
  w[2] += dz * fz;
  w[3] += dx * fy;
  w[4] += dx * fz;
  w[5] += dy * fz;
}

template <typename TF, int POT>
__device__ __forceinline__ void lj_accumulate(const LJ<TF> &lj, TF dx, TF dy, TF dz, TF r2, TF qq, TF f[3],
                                              TF &e, TF w[6]) {
  TF u;
  const TF fs = pair_terms<TF, POT>(lj, r2, qq, u);
  pair_add<TF>(dx, dy, dz, u, fs, f, e, w);
}

template <typename TF>
__device__ __forceinline__ void store_pair_out(const Sys &d, int64_t i, const TF f[3], TF e, const TF w[6]) {
  TF *F = static_cast<TF *>(d.F);
  TF *E = static_cast<TF *>(d.epot);
  TF *W = static_cast<TF *>(d.W);
  const int64_t n = d.n;
#pragma unroll
  for (int a = 0; a < 3; ++a) F[a * n + i] = f[a];
  E[i] = TF(0.5) * e;
#pragma unroll
  for (int a = 0; a < 6; ++a) W[a * n + i] = TF(0.5) * w[a];
}

__device__ __forceinline__ void image_offset(int code, int &ox, int &oy, int &oz) {
  ox = code % 3 - 1;
  oy = (code / 3) % 3 - 1;
  oz = code / 9 - 1;
}

// The displacement r_i - r_j along one axis from double-float offsets
// (hi + lo) in cells o edges apart (edge eh + el), rounded to FP32 once: the
// high words' difference is split into its rounded value and exact error
// (TwoSum), the cell offset comes off the rounded value (exact for pairs
// closer than half an edge, by Sterbenz's lemma), and the error, the low
// words and the edge's low word are added before the final rounding.
__device__ __forceinline__ float exact_disp(float hi_i, float lo_i, float hi_j, float lo_j, float o, float eh,
                                            float el) {
  const dfloat s = df_two_sum(hi_i, -hi_j);
  const float t = fmaf(-o, eh, s.h);
  const float c = fmaf(-o, el, s.l + (lo_i - lo_j));
  return t + c;
}

// Direct link-cell forces (MD_PAIR_CELLS), one warp per cell (lanes = the
// cell's atoms, 32 at a time; warps stride over the cells).  The 27
// neighbour cells are staged through shared memory 32 atoms at a time; every
// lane then sweeps the staged atoms (broadcast reads), moving each into its
// own cell's frame first (pj + o edge).  In the mixed form pairs closer than
// r_close take the rounded-once displacement (exact_disp) from the offsets'
// low words.
template <typename TF, int POT>
__global__ void __launch_bounds__(kCellWarps * 32) k_cells(Sys d, LJ<TF> lj) {
  using V4 = typename Vec4<TF>::type;
  constexpr bool kMixed = std::is_same<TF, float>::value;
  __shared__ V4 spos[kCellWarps][32];
  __shared__ float4 slo[kCellWarps][32];
  __shared__ int sidx[kCellWarps][32];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const V4 *rel = static_cast<const V4 *>(d.rel);
  for (int64_t c = blockIdx.x * (int64_t)kCellWarps + wl; c < d.ncell; c += (int64_t)gridDim.x * kCellWarps) {
    const Rep &R = d.rep[d.rep_of_cell[c]];
    const int nc = R.nc;
    const TF edge = (TF)R.edge;
    const int64_t lc = c - R.cell0;
    const int cx = (int)(lc % nc), cy = (int)((lc / nc) % nc), cz = (int)(lc / ((int64_t)nc * nc));
    const int i0 = d.cellstart[c], i1 = d.cellstart[c + 1];
    for (int ib = i0; ib < i1; ib += 32) {
      const int i = ib + lane;
      const bool act = i < i1;
      V4 pi;
      float4 li = make_float4(0.f, 0.f, 0.f, 0.f);
      if (act) {
        pi = Vec4<TF>::load(rel + i);
        if constexpr (kMixed) li = d.rlo[i];
      }
      TF f[3] = {0, 0, 0}, e = 0, w[6] = {0, 0, 0, 0, 0, 0};
      for (int code = 0; code < 27; ++code) {
        int ox, oy, oz;
        image_offset(code, ox, oy, oz);
        const int jx = (cx + ox + nc) % nc, jy = (cy + oy + nc) % nc, jz = (cz + oz + nc) % nc;
        const int64_t cj = R.cell0 + ((int64_t)jz * nc + jy) * nc + jx;
        const int j0 = d.cellstart[cj], j1 = d.cellstart[cj + 1];
        const TF offx = ox * edge, offy = oy * edge, offz = oz * edge;
        for (int jb = j0; jb < j1; jb += 32) {
          __syncwarp();
          if (jb + lane < j1) {
            spos[wl][lane] = Vec4<TF>::load(rel + jb + lane);
            if constexpr (kMixed) slo[wl][lane] = d.rlo[jb + lane];
            sidx[wl][lane] = jb + lane;
          }
          __syncwarp();
          const int nj = min(32, j1 - jb);
          if (act) {
            for (int t = 0; t < nj; ++t) {
              const V4 pj = spos[wl][t];
              // j moved into i's cell frame first: for a close pair across a
              // cell face pj + o lands next to pi, so the subtraction is exact
              TF dx = pi.x - (pj.x + offx);
              TF dy = pi.y - (pj.y + offy);
              TF dz = pi.z - (pj.z + offz);
              TF r2 = dx * dx + dy * dy + dz * dz;
              if (r2 < lj.rc2 && sidx[wl][t] != i) {
                if constexpr (kMixed) {
                  if (r2 < lj.rclose2) {
                    const float4 lj4 = slo[wl][t];
                    dx = exact_disp(pi.x, li.x, pj.x, lj4.x, (float)ox, R.edge_h, R.edge_l);
                    dy = exact_disp(pi.y, li.y, pj.y, lj4.y, (float)oy, R.edge_h, R.edge_l);
                    dz = exact_disp(pi.z, li.z, pj.z, lj4.z, (float)oz, R.edge_h, R.edge_l);
                    r2 = dx * dx + dy * dy + dz * dz;
                  }
                }
                lj_accumulate<TF, POT>(lj, dx, dy, dz, r2, pi.w * pj.w, f, e, w);
              }
            }
          }
        }
      }
      if (act) store_pair_out<TF>(d, i, f, e, w);
    }
  }
}

// Verlet-list build, one warp per chunk of 32 consecutive atoms of the
// cell-sorted order; the lists of a chunk fill one block of maxnb rows x 32
// lanes (slot k of atom i at block(i / 32) + 32 k + i % 32), so the pair
// kernel reads a row of 128 bytes per step of its loop and the rows being
// written stay together in L2.  The chunk's atoms fall into one or a few
// cells ("segments").  For each segment, j-parallel: the chunk's i
// coordinates sit in shared memory; the lanes take 32 candidate atoms at a
// time from a row of three x-adjacent neighbour cells (one contiguous range
// of the sorted order unless the row wraps), move them into the i cell's
// frame and, for each i of the segment, test all 32 at once; a ballot and a
// population count give every accepted j its list slot.
template <typename TF, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_build(Sys d, LJ<TF> lj) {
  using V4 = typename Vec4<TF>::type;
  if (!any_rebuild(d)) return;
  __shared__ V4 spi[WARPS][32];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int64_t n = d.n;
  const V4 *rel = static_cast<const V4 *>(d.rel);
  const unsigned below = (1u << lane) - 1u;
  const int64_t nchunks = (n + 31) / 32;
  for (int64_t q = blockIdx.x * (int64_t)WARPS + wl; q < nchunks; q += (int64_t)gridDim.x * WARPS) {
    const int a0 = (int)(q * 32), a1 = (int)min((int64_t)a0 + 32, n);
    __syncwarp();
    if (a0 + lane < a1) spi[wl][lane] = Vec4<TF>::load(rel + a0 + lane);
    __syncwarp();
    uint32_t *blk = d.nbr + q * d.maxnb * 32;
    int cnt = 0;  // lane l: list length of atom a0 + l
    int s = a0;
    while (s < a1) {
      // the segment: atoms of s's cell within the chunk (one replica)
      const Rep &R = rep_of(d, s);
      const int nc = R.nc;
      const TF edge = (TF)R.edge;
      int cx, cy, cz;
      unpack_cell(d.cpk[s], cx, cy, cz);
      const int e = min(d.cellstart[R.cell0 + (cz * nc + cy) * nc + cx + 1], a1);
      if (!rebuilds(d, d.rep_of_atom[s])) {  // this replica keeps its lists
        s = e;
        continue;
      }
      for (int row = 0; row < 9; ++row) {
        const int oy = row % 3 - 1, oz = row / 3 - 1;
        const int jy = (cy + oy + nc) % nc, jz = (cz + oz + nc) % nc;
        const int64_t rb = R.cell0 + ((int64_t)jz * nc + jy) * nc;
        const bool contig = cx >= 1 && cx <= nc - 2;
        for (int piece = 0; piece < (contig ? 1 : 3); ++piece) {
          int ra, rbnd, b1, b2;
          if (contig) {  // cells cx-1, cx, cx+1 of the row are contiguous
            ra = d.cellstart[rb + cx - 1];
            rbnd = d.cellstart[rb + cx + 2];
            b1 = d.cellstart[rb + cx];
            b2 = d.cellstart[rb + cx + 1];
          } else {
            const int ox = piece - 1;
            const int jx = (cx + ox + nc) % nc;
            ra = d.cellstart[rb + jx];
            rbnd = d.cellstart[rb + jx + 1];
            b1 = ox == -1 ? rbnd : ra;  // every j of this cell gets offset ox
            b2 = ox == 1 ? ra : rbnd;
          }
          for (int jb = ra; jb < rbnd; jb += 32) {
            const int j = jb + lane;
            const bool jv = j < rbnd;
            const int ox = j < b1 ? -1 : (j < b2 ? 0 : 1);
            V4 t;
            t.x = t.y = t.z = TF(0);
            if (jv) {
              const V4 pj = Vec4<TF>::load(rel + j);
              t.x = pj.x + ox * edge;
              t.y = pj.y + oy * edge;
              t.z = pj.z + oz * edge;
            }
            const uint32_t tag = list_entry(j, ox, oy, oz);
            for (int ii = s; ii < e; ++ii) {
              const int li = ii - a0;  // lane that owns atom ii
              const V4 pi = spi[wl][li];
              const TF dx = pi.x - t.x, dy = pi.y - t.y, dz = pi.z - t.z;
              const TF r2 = dx * dx + dy * dy + dz * dz;
              const bool acc = jv && r2 < lj.rlist2 && j != ii;
              const unsigned m = __ballot_sync(0xffffffffu, acc);
              if (m) {
                const int base = __shfl_sync(0xffffffffu, cnt, li);
                const int pos = base + __popc(m & below);
                if (acc && pos < d.maxnb) blk[pos * 32 + li] = tag;
                if (lane == li) cnt += __popc(m);
              }
            }
          }
        }
      }
      s = e;
    }
    if (a0 + lane < a1 && rebuilds(d, d.rep_of_atom[a0 + lane])) d.nnb[a0 + lane] = list_count(d, cnt);
  }
}

// FP64 Verlet-list pair kernel (the comparison form and the FP64 ionic
// path): one thread per atom (cell-sorted, so a warp's neighbours overlap
// and their coordinates come from L1), full neighbour shell, no atomics.
// The list is streamed with evict-first loads; the loop is unrolled by
// kUnroll so that kUnroll index loads and then kUnroll coordinate gathers
// are in flight before the arithmetic that needs them.
constexpr int kUnroll = 4;

template <typename TF, int POT>
__device__ __forceinline__ void pair_from_entry(const LJ<TF> &lj, TF edge, uint32_t ent,
                                                const typename Vec4<TF>::type &pi,
                                                const typename Vec4<TF>::type &pj, TF f[3], TF &e, TF w[6]) {
  int ox, oy, oz;
  entry_image(ent, ox, oy, oz);
  // j moved into i's cell frame first: for a close pair across a cell face
  // pj + o lands next to pi, so the final subtraction is exact.
  const TF dx = pi.x - (pj.x + ox * edge);
  const TF dy = pi.y - (pj.y + oy * edge);
  const TF dz = pi.z - (pj.z + oz * edge);
  const TF r2 = dx * dx + dy * dy + dz * dz;
  if (r2 < lj.rc2) lj_accumulate<TF, POT>(lj, dx, dy, dz, r2, pi.w * pj.w, f, e, w);
}

template <typename TF, int POT>
__global__ void __launch_bounds__(kMaxPairThreads) k_pair_list(Sys d, LJ<TF> lj) {
  using V4 = typename Vec4<TF>::type;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= d.n) return;
  const TF edge = (TF)rep_of(d, i).edge;
  const V4 *rel = static_cast<const V4 *>(d.rel);
  const V4 pi = Vec4<TF>::load(rel + i);
  TF f[3] = {0, 0, 0}, e = 0, w[6] = {0, 0, 0, 0, 0, 0};
  const int nn = d.nnb[i];
  const uint32_t *nb = d.nbr + (i >> 5) * d.maxnb * 32 + (i & 31);
  int k = 0;
  for (; k + kUnroll <= nn; k += kUnroll) {
    uint32_t ent[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) ent[u] = __ldcs(nb + (k + u) * 32);
    V4 pj[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) pj[u] = Vec4<TF>::load(rel + entry_atom(ent[u]));
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) pair_from_entry<TF, POT>(lj, edge, ent[u], pi, pj[u], f, e, w);
  }
  for (; k < nn; ++k) {
    const uint32_t ent = __ldcs(nb + k * 32);
    const V4 pj = Vec4<TF>::load(rel + entry_atom(ent));
    pair_from_entry<TF, POT>(lj, edge, ent, pi, pj, f, e, w);
  }
  store_pair_out<TF>(d, i, f, e, w);
}

// Mixed-form Verlet-list pair kernel: one thread per atom (cell-sorted, so
// a warp's neighbours overlap and their coordinates come from L1), full
// neighbour shell, no atomics (deterministic sums), FP32 FMA work on the CUDA
// cores.  The list is streamed with evict-first loads; the loop is unrolled
// by kUnroll so that kUnroll index loads and then kUnroll coordinate gathers
// are in flight before the arithmetic.  The image offsets of the at most two
// replicas a CTA spans sit in shared memory, one vector per image code.
//
// Close pairs (closer than r_close, where |dF/dr| is largest and the FP32
// rounding of the displacement dominates the force error): the main loop
// keeps their list entries (up to kMaxClose) in a per-thread array, and
// afterwards each such pair's term is replaced by the one of the
// displacement rounded once from the double-float offsets (exact_disp): the
// thread subtracts the main loop's term, recomputed by the same code, and
// adds the exact one.  At most 48 registers (five 256-thread CTAs per SM):
// measured 1 % faster than the 59 the kernel takes unbounded.
constexpr int kMaxClose = 16;

template <int POT>
__device__ __forceinline__ bool mixed_term(const LJ<float> &lj, float dx, float dy, float dz, float qq, float sign,
                                           float f[3], float &e, float w[6]) {
  const float r2 = dx * dx + dy * dy + dz * dz;
  if (r2 < lj.rc2) {
    float u;
    const float fs = pair_terms<float, POT>(lj, r2, qq, u);
    pair_add<float>(dx, dy, dz, sign * u, sign * fs, f, e, w);
  }
  return r2 < lj.rclose2;
}

template <int POT>
__global__ void __launch_bounds__(kMaxPairThreads, 5) k_pair_mixed(Sys d, LJ<float> lj) {
  __shared__ float4 offs[2][64];  // by image code (entry bits 0..5)
  const int64_t blk0 = blockIdx.x * (int64_t)blockDim.x;
  const int r0 = d.rep_of_atom[blk0];
  const int r1 = d.rep_of_atom[min(blk0 + blockDim.x, d.n) - 1];
  for (int t = threadIdx.x; t < 128; t += blockDim.x) {
    const int which = t >> 6, code = t & 63;
    const float edge = d.rep[which ? r1 : r0].edge_h;
    const int ox = (code & 3) - 1, oy = ((code >> 2) & 3) - 1, oz = ((code >> 4) & 3) - 1;
    offs[which][code] = make_float4(ox * edge, oy * edge, oz * edge, 0.f);
  }
  __syncthreads();
  const int64_t i = blk0 + threadIdx.x;
  if (i >= d.n) return;
  const int ri = d.rep_of_atom[i];
  const float4 *off = offs[ri == r0 ? 0 : 1];
  const float4 *rel = static_cast<const float4 *>(d.rel);
  const float4 pi = rel[i];
  float f[3] = {0.f, 0.f, 0.f}, e = 0.f, w[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int nn = d.nnb[i];
  const uint32_t *nb = d.nbr + (i >> 5) * d.maxnb * 32 + (i & 31);
  // j moved into i's cell frame first: for a close pair across a cell face
  // pj + o lands next to pi, so the final subtraction is exact
  auto disp = [&](uint32_t ent, const float4 &pj, float &dx, float &dy, float &dz) {
    const float4 o = off[ent & 63u];
    dx = pi.x - (pj.x + o.x);
    dy = pi.y - (pj.y + o.y);
    dz = pi.z - (pj.z + o.z);
  };
  uint32_t close[kMaxClose];
  int ncl = 0;
  int k = 0;
  for (; k + kUnroll <= nn; k += kUnroll) {
    uint32_t ent[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) ent[u] = __ldcs(nb + (k + u) * 32);
    float4 pj[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) pj[u] = rel[entry_atom(ent[u])];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      float dx, dy, dz;
      disp(ent[u], pj[u], dx, dy, dz);
      if (mixed_term<POT>(lj, dx, dy, dz, pi.w * pj[u].w, 1.f, f, e, w) && ncl < kMaxClose) close[ncl++] = ent[u];
    }
  }
  for (; k < nn; ++k) {
    const uint32_t ent = __ldcs(nb + k * 32);
    const float4 pj = rel[entry_atom(ent)];
    float dx, dy, dz;
    disp(ent, pj, dx, dy, dz);
    if (mixed_term<POT>(lj, dx, dy, dz, pi.w * pj.w, 1.f, f, e, w) && ncl < kMaxClose) close[ncl++] = ent;
  }
  if (ncl > 0) {
    const Rep &R = d.rep[ri];
    const float4 li = d.rlo[i];
    for (int c = 0; c < ncl; ++c) {
      const uint32_t ent = close[c];
      const int j = entry_atom(ent);
      const float4 pj = rel[j];
      const float4 lj4 = d.rlo[j];
      float dx, dy, dz;
      disp(ent, pj, dx, dy, dz);
      mixed_term<POT>(lj, dx, dy, dz, pi.w * pj.w, -1.f, f, e, w);
      float ox, oy, oz;
      entry_image_f(ent, ox, oy, oz);
      dx = exact_disp(pi.x, li.x, pj.x, lj4.x, ox, R.edge_h, R.edge_l);
      dy = exact_disp(pi.y, li.y, pj.y, lj4.y, oy, R.edge_h, R.edge_l);
      dz = exact_disp(pi.z, li.z, pj.z, lj4.z, oz, R.edge_h, R.edge_l);
      mixed_term<POT>(lj, dx, dy, dz, pi.w * pj.w, 1.f, f, e, w);
    }
  }
  store_pair_out<float>(d, i, f, e, w);
}

// ------------------------------------------ tile windows (MD_PAIR_TILES)
//
// Mixed-form Lennard-Jones pairs over shared-memory windows.  A replica's
// cells are cut into tiles of at most kTileExt cells per axis (segments of
// nearly equal length that never wrap); a tile's window is its cells plus
// the one-cell shell around them, (bx+2)(by+2)(bz+2) cells enumerated
// z-major, then y, then x, so the three x-neighbours of a cell are three
// consecutive window cells whose atoms fill one contiguous slot range.  The
// CTA of a tile stages every window atom in shared memory once per launch:
// its coordinate in the tile's own frame (origin at the tile centre, so
// |X| < 8 and the FP32 word keeps a resolution of 2^-21; the shell's
// periodic images come out right by construction) as a float4 X_h, and the
// double-float remainder X_l = x - X_h as three halves scaled by 2^20
// (|X_l| < 2^-20, kept to ~2^-31 absolute).  Slot 0 holds a dummy atom 10^9
// away, the padding entry of the lists.
//
// An atom's Verlet list holds the byte offsets (16 bits: slots < 4096) of
// its neighbours' slots in two segments: close entries (within r_close +
// skin at the build, so possibly within r_close before the next build),
// evaluated from the double-float coordinates with the displacement rounded
// once, and far entries, evaluated from X_h alone, two per 32-bit word and
// padded with dummies to a multiple of four.  The pair loop reads its
// neighbours from shared memory (no global gathers, no image offsets) and
// streams its list words with one block of lookahead.
constexpr int kTileExt[3] = {3, 2, 2};  // largest tile extent along x, y, z (cells)
constexpr int kMaxWinCells = 128;       // (3+2)^3 = 125 for tiles up to 3 x 3 x 3
constexpr int kMaxTileRows = 9;
constexpr int kMaxCloseT = 16;  // two blocks of eight
constexpr int kWinMaxSlots = 4096;
constexpr int kWinPad = 32;  // slots past the capacity that the build's 32-slot test batches may read
constexpr int kTileThreadsMax = 384;
constexpr float kLoScale = 1048576.f;  // 2^20
constexpr float kLoUnscale = 1.f / 1048576.f;

// Dynamic shared memory of the tile kernels: X_h [wcap + kWinPad] float4,
// then (pair kernel) X_l [wcap + kWinPad] uint2, then the window cell of
// every slot [wcap + kWinPad] bytes.
__host__ __device__ constexpr size_t tile_smem(int wcap, bool lo) {
  return (size_t)(wcap + kWinPad) * (sizeof(float4) + (lo ? sizeof(uint2) : 0) + 1);
}

// Window of one tile (shared memory).
struct TileWin {
  int WX, WY, WZ, nwc;          // window extent in cells, window cells
  int natoms, nrows, bx, by;    // atoms of the tile (-1: window over capacity), its (y, z) rows, extent
  int wsum[kMaxWinCells / 32];  // scan scratch
  int pre[kMaxWinCells + 1];    // first slot of each window cell (pre[nwc]: end)
  int gs[kMaxWinCells];         // sorted index of each window cell's first atom
  int cxyz[kMaxWinCells];       // window-cell coordinates wx | wy << 4 | wz << 8
  float ch[3][5], cl[3][5];     // tile-frame centre of the k-th window cell along each axis (hi, lo)
  int rpre[kMaxTileRows + 1];   // tile rows: prefix of their atom counts
  int rslot[kMaxTileRows];      // first slot of each row
  int rg[kMaxTileRows];         // sorted index of each row's first atom
};

__device__ __forceinline__ uint2 pack_lo(float x, float y, float z) {
  const __half2 a = __floats2half2_rn(x * kLoScale, y * kLoScale);
  const __half2 b = __floats2half2_rn(z * kLoScale, 0.f);
  return make_uint2(*reinterpret_cast<const unsigned *>(&a), *reinterpret_cast<const unsigned *>(&b));
}
__device__ __forceinline__ float3 unpack_lo(uint2 u) {
  const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
  return make_float3(a.x * kLoUnscale, a.y * kLoUnscale, b.x * kLoUnscale);
}

// 128- and 64-bit shared loads at a shared-window byte address (the
// compiler would narrow a float4 whose w goes unused into two loads).
__device__ __forceinline__ float4 lds4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ uint2 lds2(uint32_t a) {
  uint2 v;
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
  return v;
}

// Exact rounding error of s = fl(a + b) (Knuth's TwoSum).
__device__ __forceinline__ float two_sum_err(float a, float b, float s) {
  const float bb = s - a;
  return (a - (s - bb)) + (b - bb);
}

// Window layout of tile tl (every thread of the CTA calls it): a prefix sum
// over the window cells gives every cell its slot range, every slot learns
// its cell in a byte map, and thread 0 lists the tile's rows.  False when
// the window exceeds d.wcap slots (the error word is set, natoms = -1).
// The layout depends only on the cell sort, so the list build computes it
// and keeps it for the pair kernel until the next rebuild.
__device__ bool window_layout(const Sys &d, const Tile &tl, TileWin &W, unsigned char *cellof) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const Rep &R = d.rep[tl.rep];
  const int nc = R.nc;
  const int WX = tl.bx + 2, WY = tl.by + 2, WZ = tl.bz + 2, nwc = WX * WY * WZ;
  if (t < 15) {  // window-cell centres: axis t / 5, window index t % 5
    const int a = t / 5, k = t % 5;
    const int ext = a == 0 ? tl.bx : (a == 1 ? tl.by : tl.bz);
    const float m = (float)(2 * k - 1 - ext);  // half edges from the tile centre
    const float hh = 0.5f * R.edge_h;
    const float c = m * hh;
    W.ch[a][k] = c;
    W.cl[a][k] = fmaf(m, hh, -c) + m * (0.5f * R.edge_l);
  }
  int cnt = 0, incl = 0;
  if (t < kMaxWinCells) {
    if (t < nwc) {
      const int wx = t % WX, wy = (t / WX) % WY, wz = t / (WX * WY);
      int gx = tl.x0 - 1 + wx, gy = tl.y0 - 1 + wy, gz = tl.z0 - 1 + wz;
      gx += gx < 0 ? nc : (gx >= nc ? -nc : 0);
      gy += gy < 0 ? nc : (gy >= nc ? -nc : 0);
      gz += gz < 0 ? nc : (gz >= nc ? -nc : 0);
      const int64_t g = R.cell0 + ((int64_t)gz * nc + gy) * nc + gx;
      const int s0 = d.cellstart[g];
      cnt = d.cellstart[g + 1] - s0;
      W.gs[t] = s0;
      W.cxyz[t] = wx | (wy << 4) | (wz << 8);
    }
    incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) W.wsum[warp] = incl;
  }
  __syncthreads();
  if (t < kMaxWinCells) {
    int off = 0;
    for (int w = 0; w < warp; ++w) off += W.wsum[w];
    if (t < nwc) W.pre[t] = 1 + off + incl - cnt;
    if (t == nwc - 1) W.pre[nwc] = 1 + off + incl;
  }
  __syncthreads();
  const bool fail = W.pre[nwc] > d.wcap;
  if (t == 0) {
    W.WX = WX;
    W.WY = WY;
    W.WZ = WZ;
    W.nwc = nwc;
    W.bx = tl.bx;
    W.by = tl.by;
    int acc = 0, q = 0;
    for (int zq = 1; zq <= tl.bz; ++zq)
      for (int yq = 1; yq <= tl.by; ++yq, ++q) {
        const int c = (zq * WY + yq) * WX + 1;
        W.rslot[q] = W.pre[c];
        W.rg[q] = W.gs[c];
        W.rpre[q] = acc;
        acc += W.pre[c + tl.bx] - W.pre[c];
      }
    W.rpre[q] = acc;
    W.nrows = q;
    W.natoms = acc;
    if (fail) {
      atomicOr(d.err, ERR_WINDOW);
      W.natoms = -1;
    }
  }
  if (!fail && t < nwc)
    for (int s = W.pre[t], e = W.pre[t + 1]; s < e; ++s) cellof[s] = (unsigned char)t;
  __syncthreads();
  return !fail;  // uniform: every thread read the same pre[nwc]
}

// Coordinates of every window slot in the tile frame (X_h, and with LO the
// remainder X_l), from the layout in W and cellof; slot 0 gets the dummy.
// Each thread handles its slots three at a time, so that their coordinate
// loads are in flight together.
template <bool LO>
__device__ void stage_coords(const Sys &d, const TileWin &W, float4 *whi, uint2 *wlo, const unsigned char *cellof) {
  const int t = threadIdx.x;
  const float4 *rel = static_cast<const float4 *>(d.rel);
  const int end = W.pre[W.nwc], T = blockDim.x;
  constexpr int U = 3;
  for (int s0 = 1 + t; s0 < end; s0 += U * T) {
    int jj[U], xyz[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int s = s0 + u * T;
      const int c = s < end ? cellof[s] : 0;
      jj[u] = W.gs[c] + (s - W.pre[c]);
      xyz[u] = W.cxyz[c];
    }
    float4 h[U], l[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (s0 + u * T < end) {
        h[u] = rel[jj[u]];
        if constexpr (LO) l[u] = d.rlo[jj[u]];
      }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int s = s0 + u * T;
      if (s < end) {
        const int kx = xyz[u] & 15, ky = (xyz[u] >> 4) & 15, kz = xyz[u] >> 8;
        const float cx = W.ch[0][kx], cy = W.ch[1][ky], cz = W.ch[2][kz];
        const float xh = cx + h[u].x, yh = cy + h[u].y, zh = cz + h[u].z;
        whi[s] = make_float4(xh, yh, zh, 0.f);
        if constexpr (LO)
          wlo[s] = pack_lo(two_sum_err(cx, h[u].x, xh) + (W.cl[0][kx] + l[u].x),
                           two_sum_err(cy, h[u].y, yh) + (W.cl[1][ky] + l[u].y),
                           two_sum_err(cz, h[u].z, zh) + (W.cl[2][kz] + l[u].z));
      }
    }
  }
  if (t == 0) {
    whi[0] = make_float4(1e9f, 1e9f, 1e9f, 0.f);
    if constexpr (LO) wlo[0] = make_uint2(0u, 0u);
  }
  __syncthreads();
}

// The t-th atom of the tile: its sorted index i, its slot wi and its window
// cell (wx, wy, wz).
__device__ __forceinline__ void tile_atom(const TileWin &W, int t, int64_t &i, int &wi, int &wx, int &wy, int &wz) {
  int q = 0;
  while (q + 1 < W.nrows && W.rpre[q + 1] <= t) ++q;
  const int k = t - W.rpre[q];
  wi = W.rslot[q] + k;
  i = W.rg[q] + k;
  wy = q % W.by + 1;
  wz = q / W.by + 1;
  const int c = (wz * W.WY + wy) * W.WX;
  wx = 1;
  while (wx < W.bx && W.pre[c + wx + 1] <= wi) ++wx;
}

// Appends a 16-bit entry to four words that fill up as one block of eight
// (entry k in bits 16k.. of the 128 bits): every word moves down by one
// entry and the new one comes in at the top.
__device__ __forceinline__ void push16(uint32_t (&w)[4], uint32_t off) {
  w[0] = __funnelshift_r(w[0], w[1], 16);
  w[1] = __funnelshift_r(w[1], w[2], 16);
  w[2] = __funnelshift_r(w[2], w[3], 16);
  w[3] = __funnelshift_r(w[3], off, 16);
}

// gm |= bit when r2 < lim (a predicated OR: no branch, so the lanes of a
// warp never split over a distance test).
__device__ __forceinline__ void or_if_less(uint32_t &gm, float r2, float lim, uint32_t bit) {
  asm("{\n\t.reg .pred p;\n\tsetp.lt.f32 p, %1, %2;\n\t@p or.b32 %0, %0, %3;\n\t}"
      : "+r"(gm)
      : "f"(r2), "f"(lim), "r"(bit));
}

__device__ __forceinline__ float dist2(const float4 &a, const float4 &b) {
  const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  return dx * dx + dy * dy + dz * dz;
}

// List build of the tiles whose replica rebuilds: every atom of the tile
// against the 27 window cells around its own (nine contiguous slot ranges
// of three cells), 32 slots at a time.  The distance tests (groups of eight,
// predicated) fill two bit masks, within r_list and within the close radius
// r_close + skin, before anything is appended; the accepted slots are then
// appended in warp-uniform loops (as many rounds as the lane with the most
// entries needs), close entries first.  Entries leave as blocks of eight in
// slot order, the last block of each segment padded with the dummy slot 0.
__global__ void __launch_bounds__(kTileThreadsMax, 2) k_build_tile(Sys d, LJ<float> lj) {
  if (!any_rebuild(d)) return;
  const Tile tl = d.tiles[blockIdx.x];
  if (!rebuilds(d, tl.rep)) return;
  extern __shared__ float4 whi[];
  unsigned char *cellof = reinterpret_cast<unsigned char *>(whi + d.wcap + kWinPad);
  __shared__ TileWin W;
  const bool ok = window_layout(d, tl, W, cellof);
  {  // the layout, kept for the pair kernel until the next rebuild
    const int *src = reinterpret_cast<const int *>(&W);
    int *dst = reinterpret_cast<int *>(d.trec + blockIdx.x);
    for (int k = threadIdx.x; k < (int)(sizeof(TileWin) / 4); k += blockDim.x) dst[k] = src[k];
    const uint4 *cs = reinterpret_cast<const uint4 *>(cellof);
    uint4 *cd = reinterpret_cast<uint4 *>(d.tcell + (int64_t)blockIdx.x * (d.wcap + kWinPad));
    if (ok)
      for (int k = threadIdx.x; k < (d.wcap + kWinPad) / 16; k += blockDim.x) cd[k] = cs[k];
  }
  if (!ok) return;
  stage_coords<false>(d, W, whi, nullptr, cellof);
  const uint32_t wbase = (uint32_t)__cvta_generic_to_shared(whi);
  const int64_t n = d.n;
  const int maxb = d.maxnb >> 3;
  for (int t = threadIdx.x; t < W.natoms; t += blockDim.x) {
    int64_t i;
    int wi, wx, wy, wz;
    tile_atom(W, t, i, wi, wx, wy, wz);
    const float4 xi = whi[wi];
    uint4 *far = d.tnb + i;
    uint4 *cl = d.tcl + i;
    uint32_t fw[4] = {0u, 0u, 0u, 0u}, cw[4] = {0u, 0u, 0u, 0u};
    int nfar = 0, ncl = 0;
    auto put_far = [&](uint32_t off) {
      push16(fw, off);
      if ((++nfar & 7) == 0 && (nfar >> 3) <= maxb)
        far[(int64_t)((nfar >> 3) - 1) * n] = make_uint4(fw[0], fw[1], fw[2], fw[3]);
    };
    for (int row = 0; row < 9; ++row) {
      const int c = ((wz + row / 3 - 1) * W.WY + (wy + row % 3 - 1)) * W.WX + wx - 1;
      const int s1 = W.pre[c + 3];
      for (int s = W.pre[c]; s < s1; s += 32) {
        const uint32_t a0 = wbase + ((uint32_t)s << 4);
        const int m = min(32, s1 - s);
        uint32_t am = 0u, cm = 0u;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          if (8 * g < m) {
            uint32_t ga = 0u, gc = 0u;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const float r2 = dist2(xi, lds4(a0 + 16u * (8 * g + u)));
              or_if_less(ga, r2, lj.rlist2, 1u << u);
              or_if_less(gc, r2, lj.rcb2, 1u << u);
            }
            am |= ga << (8 * g);
            cm |= gc << (8 * g);
          }
        }
        if (m < 32) am &= (1u << m) - 1u;
        const int self = wi - s;
        if (self >= 0 && self < 32) am &= ~(1u << self);
        cm &= am;
        uint32_t fm = am & ~cm;
        const unsigned act = __activemask();
        const int mc = __reduce_max_sync(act, __popc(cm));
        for (int k = 0; k < mc; ++k) {
          if (cm) {
            const int b = __ffs(cm) - 1;
            cm &= cm - 1u;
            if (ncl < kMaxCloseT) {
              push16(cw, (uint32_t)(s + b) << 4);
              if ((++ncl & 7) == 0) cl[(int64_t)((ncl >> 3) - 1) * n] = make_uint4(cw[0], cw[1], cw[2], cw[3]);
            } else {
              fm |= 1u << b;  // beyond the close capacity: FP32 displacement
            }
          }
        }
        const int mf = __reduce_max_sync(act, __popc(fm));
        for (int k = 0; k < mf; ++k) {
          if (fm) {
            const int b = __ffs(fm) - 1;
            fm &= fm - 1u;
            put_far((uint32_t)(s + b) << 4);
          }
        }
      }
    }
    if (ncl & 7) {  // pad the last close block with the dummy
      const int pad = 8 - (ncl & 7);
      for (int k = 0; k < pad; ++k) push16(cw, 0u);
      cl[(int64_t)(ncl >> 3) * n] = make_uint4(cw[0], cw[1], cw[2], cw[3]);
    }
    while (nfar & 7) put_far(0u);
    d.nnb[i] = list_count(d, nfar) | (ncl << 16);
  }
}

// One far or close term, branch-free (out of range: ir2 = 0, so every
// accumulated product is 0); the energy shift is applied once per atom from
// the count of pairs in range.
__device__ __forceinline__ void tile_term(const LJ<float> &lj, float dx, float dy, float dz, float f[3], float &e,
                                          float w[6], int &cnt) {
  const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  const float rr = pair_rcp(r2);
  float ir2;  // rr in range, else 0; cnt counts the pairs in range (predicated, no branch)
  asm("{\n\t.reg .pred p;\n\tsetp.lt.f32 p, %2, %3;\n\tselp.f32 %0, %4, 0f00000000, p;\n\t@p add.s32 %1, %1, 1;\n\t}"
      : "=f"(ir2), "+r"(cnt)
      : "f"(r2), "f"(lj.rc2), "f"(rr));
  const float ir6 = ir2 * ir2 * ir2;
  e = fmaf(ir6, fmaf(lj.c12, ir6, -lj.c6), e);
  const float fs = ir2 * ir6 * fmaf(lj.f12, ir6, -lj.f6);
  const float fx = fs * dx, fy = fs * dy, fz = fs * dz;
  f[0] += fx;
  f[1] += fy;
  f[2] += fz;
  w[0] = fmaf(dx, fx, w[0]);
  w[1] = fmaf(dy, fy, w[1]);
  w[2] = fmaf(dz, fz, w[2]);
  w[3] = fmaf(dx, fy, w[3]);
  w[4] = fmaf(dx, fz, w[4]);
  w[5] = fmaf(dy, fz, w[5]);
}

// The displacement a - b of two double-float coordinates, rounded once.
__device__ __forceinline__ float df_disp(float ah, float al, float bh, float bl) {
  const dfloat s = df_two_sum(ah, -bh);
  return s.h + (s.l + (al - bl));
}

// Pair forces, per-particle energies and virials of one tile per CTA.  The
// list blocks are streamed two ahead (the close block and the first two far
// blocks are requested before any arithmetic).
__global__ void __launch_bounds__(kTileThreadsMax, 3) k_pair_tile(Sys d, LJ<float> lj) {
  extern __shared__ float4 whi[];
  uint2 *wlo = reinterpret_cast<uint2 *>(whi + d.wcap + kWinPad);
  unsigned char *cellof = reinterpret_cast<unsigned char *>(wlo + d.wcap + kWinPad);
  __shared__ TileWin W;
  {  // the layout the last list build kept (one coalesced load)
    const int *src = reinterpret_cast<const int *>(d.trec + blockIdx.x);
    int *dst = reinterpret_cast<int *>(&W);
    for (int k = threadIdx.x; k < (int)(sizeof(TileWin) / 4); k += blockDim.x) dst[k] = src[k];
    const uint4 *cs = reinterpret_cast<const uint4 *>(d.tcell + (int64_t)blockIdx.x * (d.wcap + kWinPad));
    uint4 *cd = reinterpret_cast<uint4 *>(cellof);
    for (int k = threadIdx.x; k < (d.wcap + kWinPad) / 16; k += blockDim.x) cd[k] = cs[k];
  }
  __syncthreads();
  if (W.natoms < 0) return;  // the build found the window over capacity (error word set)
  stage_coords<true>(d, W, whi, wlo, cellof);
  const uint32_t wbase = (uint32_t)__cvta_generic_to_shared(whi);
  const uint32_t lbase = (uint32_t)__cvta_generic_to_shared(wlo);
  const int64_t n = d.n;
  float *F = static_cast<float *>(d.F);
  float *E = static_cast<float *>(d.epot);
  float *Wv = static_cast<float *>(d.W);
  const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
  for (int t = threadIdx.x; t < W.natoms; t += blockDim.x) {
    int64_t i;
    int wi, wx, wy, wz;
    tile_atom(W, t, i, wi, wx, wy, wz);
    const int nn = d.nnb[i];
    const int nb = (nn & 0xffff) >> 3, ncl = nn >> 16;
    const uint4 *lw = d.tnb + i;
    const uint4 *lc = d.tcl + i;
    const uint4 C0 = ncl > 0 ? __ldcs(lc) : zero;
    uint4 A = nb > 0 ? __ldcs(lw) : zero;
    uint4 B = nb > 1 ? __ldcs(lw + n) : zero;
    const float4 xi = whi[wi];
    const float3 li = unpack_lo(wlo[wi]);
    float f[3] = {0.f, 0.f, 0.f}, e = 0.f, w[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int cnt = 0;
    auto close_term = [&](uint32_t off) {
      const float4 pj = lds4(wbase + off);
      const float3 lj3 = unpack_lo(lds2(lbase + (off >> 1)));
      tile_term(lj, df_disp(xi.x, li.x, pj.x, lj3.x), df_disp(xi.y, li.y, pj.y, lj3.y),
                df_disp(xi.z, li.z, pj.z, lj3.z), f, e, w, cnt);
    };
    auto close_block = [&](const uint4 &q, int m) {  // the first m entries of a block
      const uint32_t v[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k < m) close_term(k & 1 ? v[k >> 1] >> 16 : v[k >> 1] & 0xffffu);
    };
    close_block(C0, ncl);
    if (ncl > 8) close_block(__ldcs(lc + n), ncl - 8);
    auto far_term = [&](uint32_t off) {
      const float4 pj = lds4(wbase + off);
      tile_term(lj, xi.x - pj.x, xi.y - pj.y, xi.z - pj.z, f, e, w, cnt);
    };
    for (int k = 0; k < nb; ++k) {
      const uint4 C = k + 2 < nb ? __ldcs(lw + (int64_t)(k + 2) * n) : zero;
      far_term(A.x & 0xffffu);
      far_term(A.x >> 16);
      far_term(A.y & 0xffffu);
      far_term(A.y >> 16);
      far_term(A.z & 0xffffu);
      far_term(A.z >> 16);
      far_term(A.w & 0xffffu);
      far_term(A.w >> 16);
      A = B;
      B = C;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) F[a * n + i] = f[a];
    E[i] = 0.5f * fmaf(-lj.ushift, (float)cnt, e);
#pragma unroll
    for (int a = 0; a < 6; ++a) Wv[a * n + i] = 0.5f * w[a];
  }
}

// ---------------------------------------------------- reduce and sample

// Second half kick, then the per-step observables of every replica
// (Sec. 2.3): K, U, V sigma_ab = sum m v_a v_b + sum W_i,ab,
// V q = sum (E_i v_i + W_i v_i).  Each CTA works on one replica (rep_of_block)
// and strides over that replica's atoms.  Per-thread partial sums: FP64 in
// the FP64 form; in the mixed form every term is formed in double-float
// arithmetic from the double-float velocity, the double-float mass and the
// FP32 per-particle energy and virial, and summed by a compensated FP32
// accumulator (dfacc), so the partials carry ~48 bits like FP64 sums of
// the same inputs; the CTA merges them in double-float too (butterflies
// across each warp, then the warps in fixed order) and converts once per
// CTA, since FP64 instructions run at a small fraction of the FP32 rate
// (the FP64 merge took 15 % of the kernel).  The replica tree is FP64
// (fixed order: deterministic).  The mixed form runs at most 64 registers,
// so four CTAs fit an SM and the ~500 CTAs of a 2,048,000-atom system run
// in one wave (measured 6 % faster than three CTAs per SM).  The last CTA
// of a replica writes its observables; the
// last replica to finish advances the step counter.  When a velocity sample
// is due, velocities are also scattered to atom-id order.  The stress,
// heat-flux and mass-flux correlator samples of the step are taken from the
// observables by k_push_scalars, a separate launch that can run beside the
// next step.
template <typename TF, typename A, bool KICK>
__global__ void __launch_bounds__(kThreads, sizeof(TF) == 4 ? 4 : 3)
    k_kick_reduce(Sys d, double hdt) {
  __shared__ double red[kThreads / 32][kNRed];
  __shared__ double tot[kNRed];
  __shared__ int last;
  const TF *F = static_cast<const TF *>(d.F);
  const TF *Ep = static_cast<const TF *>(d.epot);
  const TF *Wp = static_cast<const TF *>(d.W);
  TF *vb = static_cast<TF *>(d.vbuf);
  const int64_t n = d.n;
  const StepDev *st = d.st;
  const int64_t step_now = st->step + (KICK ? 1 : 0);
  const bool vacf_due = KICK && d.vacf_u > 0 && ((step_now - st->corr_base) % d.vacf_u == 0);
  if (vacf_due)  // this push's input slot
    vb += (((step_now - st->corr_base) / d.vacf_u - 1) % d.vacf_slots) * 3 * n;
  const int r = d.rep_of_block[blockIdx.x];
  const Rep &R = d.rep[r];
  const int lb = (int)(blockIdx.x - R.block0);
  if constexpr (std::is_same<TF, float>::value) {
    dfacc acc[kNRed + 3];  // [kNRed, kNRed + 3): the virial diagonal (sigma's kinetic diagonal in [2, 5))
    const bool unit_mass = d.unit_mass != 0;
    for (int64_t i = R.atom0 + (int64_t)lb * blockDim.x + threadIdx.x; i < R.atom1;
         i += (int64_t)R.nblk * blockDim.x) {
      // every load of the atom first (the stores below could alias them)
      const int t = type_of(d, i);
      const float ep = Ep[i];
      float w[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) w[q] = Wp[q * n + i];
      float f[3], vh[3], vl[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        f[a] = KICK ? F[a * n + i] : 0.f;
        vh[a] = d.vh[a * n + i];
        vl[a] = d.vl[a * n + i];
      }
      const int id = vacf_due ? d.id[i] : 0;
      const dfloat h{d.hdtm_h[t], d.hdtm_l[t]};
      dfloat v[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        v[a] = dfloat{vh[a], vl[a]};
        if (KICK) {
          v[a] = df_add(v[a], df_mul_f(h, f[a]));
          d.vh[a * n + i] = v[a].h;
          d.vl[a * n + i] = v[a].l;
        }
      }
      if (vacf_due) {
#pragma unroll
        for (int a = 0; a < 3; ++a) vb[a * n + id] = v[a].h;
      }
      const dfloat m{d.mass_h[t], d.mass_l[t]};
      dfloat mv[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) mv[a] = unit_mass ? v[a] : df_prod(m, v[a]);
      // m v_a v_b in the order xx yy zz xy xz yz of sigma and W
      const dfloat mvv[6] = {df_prod(mv[0], v[0]), df_prod(mv[1], v[1]), df_prod(mv[2], v[2]),
                             df_prod(mv[0], v[1]), df_prod(mv[0], v[2]), df_prod(mv[1], v[2])};
      // E_i = m v^2 / 2 + epot_i, kept as an unnormalised pair
      dfloat E;
      {
        const dfloat s1 = df_two_sum(mvv[0].h, mvv[1].h);
        const dfloat s2 = df_two_sum(s1.h, mvv[2].h);
        const dfloat s3 = df_two_sum(0.5f * s2.h, ep);
        E = dfloat{s3.h, s3.l + 0.5f * (s1.l + s2.l + mvv[0].l + mvv[1].l + mvv[2].l)};
      }
      // diagonal: kinetic and virial parts apart (2K is the sum of the kinetic ones)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        acc[2 + a].add(mvv[a]);
        acc[kNRed + a].add(w[a]);
      }
      acc[1].add(ep);
#pragma unroll
      for (int q = 3; q < 6; ++q) {
        acc[2 + q].add(mvv[q]);
        acc[2 + q].add(w[q]);
      }
      // ((E_i + W_aa) v_a + sum_{b != a} W_ab v_b, with W symmetric: rows
      // (xx xy xz), (xy yy yz), (xz yz zz)
      const int row[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const dfloat ew = df_two_sum(E.h, w[a]);
        acc[8 + a].add(df_prod(dfloat{ew.h, ew.l + E.l}, v[a]));
#pragma unroll
        for (int b = 0; b < 3; ++b)
          if (b != a) acc[8 + a].add(df_prod_f(w[row[a][b]], v[b]));
      }
      if (t == d.flux_species) {
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[11 + a].add(mv[a]);
      }
    }
    // the CTA's sums: double-float butterflies across each warp, then the
    // warps' results merged in fixed order (FP64 only once per CTA)
    __shared__ float2 redf[kThreads / 32][kNRed + 3];
    __shared__ double totf[kNRed + 3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 1; q < kNRed + 3; ++q) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, acc[q].s, o);
        const float c2 = __shfl_xor_sync(0xffffffffu, acc[q].c, o);
        acc[q].merge(s2, c2);
      }
      if (lane == 0) redf[warp][q] = make_float2(acc[q].s, acc[q].c);
    }
    __syncthreads();
    if (threadIdx.x >= 1 && threadIdx.x < kNRed + 3) {
      dfacc a;
      a.s = redf[0][threadIdx.x].x;
      a.c = redf[0][threadIdx.x].y;
      for (int w = 1; w < kThreads / 32; ++w) a.merge(redf[w][threadIdx.x].x, redf[w][threadIdx.x].y);
      totf[threadIdx.x] = a.value();
    }
    __syncthreads();
    if (threadIdx.x < kNRed) {
      // 2K from the kinetic diagonal, then the virial diagonal added to sigma
      const int q = threadIdx.x;
      const double v = q == 0 ? 0.5 * (totf[2] + totf[3] + totf[4])
                              : (q >= 2 && q < 5 ? totf[q] + totf[kNRed + q - 2] : totf[q]);
      d.partials[blockIdx.x * kNRed + q] = v;
    }
  } else {  // FP64 form
    A acc[kNRed];
#pragma unroll
    for (int q = 0; q < kNRed; ++q) acc[q] = A(0);
    for (int64_t i = R.atom0 + (int64_t)lb * blockDim.x + threadIdx.x; i < R.atom1;
         i += (int64_t)R.nblk * blockDim.x) {
      // every load of the atom first (the stores below could alias them for
      // the compiler), so they are all in flight together
      const int t = type_of(d, i);
      const A ep = (A)Ep[i];
      A w[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) w[q] = (A)Wp[q * n + i];
      TF f[3];
      double vv[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        f[a] = KICK ? F[a * n + i] : TF(0);
        vv[a] = d.v[a * n + i];
      }
      const int id = vacf_due ? d.id[i] : 0;
      A v[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        double va = vv[a];
        if (KICK) {
          va = fma(hdt * d.invm[t], f[a], va);
          d.v[a * n + i] = va;
        }
        v[a] = (A)va;
      }
      if (vacf_due) {
#pragma unroll
        for (int a = 0; a < 3; ++a) vb[a * n + id] = (TF)v[a];
      }
      const A m = (A)d.mass[t];
      const A vx = v[0], vy = v[1], vz = v[2];
      const A ke = A(0.5) * m * (vx * vx + vy * vy + vz * vz);
      const A E = ke + ep;
      acc[0] += ke;
      acc[1] += ep;
      acc[2] += m * vx * vx + w[0];
      acc[3] += m * vy * vy + w[1];
      acc[4] += m * vz * vz + w[2];
      acc[5] += m * vx * vy + w[3];
      acc[6] += m * vx * vz + w[4];
      acc[7] += m * vy * vz + w[5];
      acc[8] += E * vx + w[0] * vx + w[3] * vy + w[4] * vz;
      acc[9] += E * vy + w[3] * vx + w[1] * vy + w[5] * vz;
      acc[10] += E * vz + w[4] * vx + w[5] * vy + w[2] * vz;
      const A sel = t == d.flux_species ? m : A(0);
      acc[11] += sel * vx;
      acc[12] += sel * vy;
      acc[13] += sel * vz;
    }
    double part[kNRed];  // this thread's partial sums
#pragma unroll
    for (int q = 0; q < kNRed; ++q) part[q] = (double)acc[q];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kNRed; ++q) {
      const double sm = warp_sum(part[q]);
      if (lane == 0) red[warp][q] = sm;
    }
    __syncthreads();
    if (threadIdx.x < kNRed) {
      double sm = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) sm += red[w][threadIdx.x];
      d.partials[blockIdx.x * kNRed + threadIdx.x] = sm;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(d.counter + r, 1u) == (unsigned)R.nblk - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the replica's partials: thread t sums CTAs t, t + 256, ... (all kNRed
  // values at once, independent loads), then a fixed tree over the threads
  {
    double ps[kNRed];
#pragma unroll
    for (int q = 0; q < kNRed; ++q) ps[q] = 0.0;
    for (int b = threadIdx.x; b < R.nblk; b += kThreads) {
      const double *pp = d.partials + (R.block0 + b) * kNRed;
#pragma unroll
      for (int q = 0; q < kNRed; ++q) ps[q] += __ldcg(pp + q);
    }
#pragma unroll
    for (int q = 0; q < kNRed; ++q) {
      const double sm = warp_sum(ps[q]);
      if (lane == 0) red[warp][q] = sm;
    }
    __syncthreads();
    if (threadIdx.x < kNRed) {
      double sm = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) sm += red[w][threadIdx.x];
      tot[threadIdx.x] = sm;
    }
  }
  __syncthreads();
  const int64_t nr = R.atom1 - R.atom0;
  const double V = R.L * R.L * R.L;
  if (threadIdx.x == 0) {
    ObsDev *ow = d.obs + r;
    ow->K = tot[0];
    ow->U = tot[1];
    ow->T = nr > 1 ? 2.0 * tot[0] / (3.0 * (double)nr - 3.0) : 0.0;
    for (int a = 0; a < 6; ++a) ow->sigma[a] = tot[2 + a] / V;
    for (int a = 0; a < 3; ++a) ow->q[a] = tot[8 + a] / V;
    for (int a = 0; a < 3; ++a) ow->j[a] = tot[11 + a] / V;
    if (KICK) {
      ow->Tsum += ow->T;
      ow->Tn += 1;
    }
    d.counter[r] = 0u;
  }
  // the last replica to finish closes the step
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&d.st->reps_done, 1u) == (unsigned)d.nrep - 1;
  }
  __syncthreads();
  if (!last) return;
  for (int k = threadIdx.x; k <= d.nrep; k += blockDim.x) d.rebuild[k] = 0;
  if (threadIdx.x == 0) {
    d.st->reps_done = 0u;
    if (KICK) d.st->step = step_now;
  }
}

// The step's samples of the scalar correlators (Algorithm 1), one thread per
// series: replica r's stress series 3r..3r+2 (sigma_xy, sigma_xz, sigma_yz),
// heat-flux series 3r..3r+2 (q_x, q_y, q_z) and mass-flux cross series
// 6r..6r+5 ((q_a, j_a), then (j_a, j_a)), from the observables k_kick_reduce
// wrote for the step it counted.
__global__ void k_push_scalars(Sys d, CorrDev cs, int64_t us, CorrDev ch, int64_t uh, CorrDev cm, int64_t um) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= (int64_t)d.nrep * 12) return;
  const int r = (int)(k / 12), tid = (int)(k % 12);
  const ObsDev &o = d.obs[r];
  const int64_t tc = d.st->step - d.st->corr_base;
  if (tid < 3) {
    if (us > 0 && cs.b > 0 && tc % us == 0) push_one_series<double>(cs, 3 * r + tid, o.sigma[3 + tid], o.sigma[3 + tid], tc / us);
  } else if (tid < 6) {
    if (uh > 0 && ch.b > 0 && tc % uh == 0) push_one_series<double>(ch, 3 * r + tid - 3, o.q[tid - 3], o.q[tid - 3], tc / uh);
  } else if (um > 0 && cm.b > 0 && tc % um == 0) {
    const int a = (tid - 6) % 3;
    const double y = o.j[a];
    const double x = tid < 9 ? o.q[a] : y;
    push_one_series<double>(cm, 6 * r + tid - 6, x, y, tc / um);
  }
}

// Multiplies velocities by their replica's factor lam[r].
template <typename TF>
__global__ void k_scale_v(Sys d) {
  const int64_t n = d.n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double lam = d.lam[d.rep_of_atom[i % n]];
    if constexpr (std::is_same<TF, double>::value) {
      d.v[i] *= lam;
    } else {
      const dfloat v = df_mul(dfloat{d.vh[i], d.vl[i]}, df_from_double(lam));
      d.vh[i] = v.h;
      d.vl[i] = v.l;
    }
  }
}

__global__ void k_iota(int *id, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    id[i] = (int)i;
}

// Mixed form set-up: FP64 input positions and velocities (in the rB, vB
// scratch, input order) become cell index + double-float offset from the
// cell centre and double-float velocities.  FP64 arithmetic, once.
// Replica of every atom (which = 0), cell (1) or reduction CTA (2): the
// last replica whose range starts at or before the index (binary search over
// the descriptor table; the ranges are laid end to end in replica order).
__global__ void k_rep_of(const Rep *rep, int nrep, int which, int *dst, int64_t total) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nrep - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      const int64_t start = which == 0 ? rep[mid].atom0 : (which == 1 ? rep[mid].cell0 : rep[mid].block0);
      if (start <= x)
        lo = mid;
      else
        hi = mid - 1;
    }
    dst[x] = lo;
  }
}

// Sets ERR_NONFINITE when any of count values is NaN or infinite (md_init's
// check of the caller's coordinates and velocities).
__global__ void k_check_finite(const double *a, int64_t count, unsigned *err) {
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(a[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, ERR_NONFINITE);
}

__global__ void k_init_df(Sys d) {
  const int64_t n = d.n;
  float4 *rel = static_cast<float4 *>(d.rel);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const Rep &R = rep_of(d, i);
    const int nc = R.nc;
    int ci[3];
    float oh[3], ol[3];
    for (int a = 0; a < 3; ++a) {
      double x = d.rB[a * n + i];
      x -= R.L * floor(x / R.L);
      if (x >= R.L) x -= R.L;
      if (x < 0.0) x = 0.0;
      int c = (int)(x / R.edge);
      c = c < nc ? c : nc - 1;
      ci[a] = c;
      const dfloat off = df_from_double(x - (c + 0.5) * R.edge);
      oh[a] = off.h;
      ol[a] = off.l;
      const dfloat v = df_from_double(d.vB[a * n + i]);
      d.vh[a * n + i] = v.h;
      d.vl[a * n + i] = v.l;
    }
    rel[i] = make_float4(oh[0], oh[1], oh[2], (float)d.charge[type_of(d, i)]);
    d.rlo[i] = make_float4(ol[0], ol[1], ol[2], 0.f);
    d.cpk[i] = pack_cell(ci[0], ci[1], ci[2]);
  }
}

// Per-particle outputs back in atom-id order (FP64), positions wrapped into
// their replica's box.
template <typename TF>
__global__ void k_unsort(Sys d, double *r, double *v, double *F, double *epot, double *W) {
  const int64_t n = d.n;
  const TF *Fs = static_cast<const TF *>(d.F);
  const TF *Es = static_cast<const TF *>(d.epot);
  const TF *Ws = static_cast<const TF *>(d.W);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const Rep &R = rep_of(d, i);
    const int64_t id = d.id[i];
    int cc[3];
    unpack_cell(d.cpk[i], cc[0], cc[1], cc[2]);
    for (int a = 0; a < 3; ++a) {
      if (r) {
        double x;
        if constexpr (std::is_same<TF, double>::value) {
          x = d.r[a * n + i];
        } else {
          const float4 o = static_cast<const float4 *>(d.rel)[i];
          const float4 lo = d.rlo[i];
          const float oh = a == 0 ? o.x : (a == 1 ? o.y : o.z);
          const float ol = a == 0 ? lo.x : (a == 1 ? lo.y : lo.z);
          x = (cc[a] + 0.5) * R.edge + df_to_double(dfloat{oh, ol});
        }
        x -= R.L * floor(x / R.L);
        if (x >= R.L) x -= R.L;
        r[a * n + id] = x;
      }
      if (v) {
        if constexpr (std::is_same<TF, double>::value)
          v[a * n + id] = d.v[a * n + i];
        else
          v[a * n + id] = df_to_double(dfloat{d.vh[a * n + i], d.vl[a * n + i]});
      }
      if (F) F[a * n + id] = (double)Fs[a * n + i];
    }
    if (epot) epot[id] = (double)Es[i];
    if (W)
      for (int a = 0; a < 6; ++a) W[a * n + id] = (double)Ws[a * n + i];
  }
}

// Verlet-list build, staged: one warp per chunk of 32 consecutive atoms
// (the list layout of k_build).  For each segment (the chunk's atoms of one
// cell) the warp copies the candidates -- the atoms of the 27 neighbour
// cells, row by row, already moved into the segment cell's frame and tagged
// with their list entry -- into shared memory in batches of kStageBatch,
// densely packed (k_build leaves lanes idle at the end of every 3-cell
// row).  Each atom of the segment then tests a batch 32 candidates at a
// time; the running list length is warp-uniform inside a batch, so an
// append is one ballot and one population count.  Same candidates in the
// same order as k_build, so the same lists.
template <typename TF, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_build_staged(Sys d, LJ<TF> lj) {
  using V4 = typename Vec4<TF>::type;
  constexpr int kStageBatch = sizeof(TF) == 4 ? 256 : 128;  // staged candidates per warp
  if (!any_rebuild(d)) return;
  __shared__ V4 sxyz[WARPS][kStageBatch];
  __shared__ uint32_t stag[WARPS][kStageBatch];
  __shared__ V4 spi[WARPS][32];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int64_t n = d.n;
  const V4 *rel = static_cast<const V4 *>(d.rel);
  const unsigned below = (1u << lane) - 1u;
  const int64_t nchunks = (n + 31) / 32;
  for (int64_t q = blockIdx.x * (int64_t)WARPS + wl; q < nchunks; q += (int64_t)gridDim.x * WARPS) {
    const int a0 = (int)(q * 32), a1 = (int)min((int64_t)a0 + 32, n);
    __syncwarp();
    if (a0 + lane < a1) spi[wl][lane] = Vec4<TF>::load(rel + a0 + lane);
    __syncwarp();
    uint32_t *blk = d.nbr + q * d.maxnb * 32;
    int cnt = 0;  // lane l: list length of atom a0 + l
    int s = a0;
    while (s < a1) {
      const Rep &R = rep_of(d, s);
      const int nc = R.nc;
      const TF edge = (TF)R.edge;
      int cx, cy, cz;
      unpack_cell(d.cpk[s], cx, cy, cz);
      const int e = min(d.cellstart[R.cell0 + (cz * nc + cy) * nc + cx + 1], a1);
      if (!rebuilds(d, d.rep_of_atom[s])) {
        s = e;
        continue;
      }
      int fill = 0;  // candidates in the batch
      // tests the staged batch against every atom of the segment
      auto flush = [&]() {
        __syncwarp();
        for (int ii = s; ii < e; ++ii) {
          const int li = ii - a0;
          const V4 pi = spi[wl][li];
          int c0 = __shfl_sync(0xffffffffu, cnt, li);
          for (int b0 = 0; b0 < fill; b0 += 32) {
            const int k = b0 + lane;
            bool acc = false;
            uint32_t tag = 0;
            if (k < fill) {
              const V4 t = sxyz[wl][k];
              tag = stag[wl][k];
              const TF dx = pi.x - t.x, dy = pi.y - t.y, dz = pi.z - t.z;
              const TF r2 = dx * dx + dy * dy + dz * dz;
              acc = r2 < lj.rlist2 && entry_atom(tag) != ii;
            }
            const unsigned m = __ballot_sync(0xffffffffu, acc);
            const int pos = c0 + __popc(m & below);
            if (acc && pos < d.maxnb) blk[pos * 32 + li] = tag;
            c0 += __popc(m);
          }
          if (lane == li) cnt = c0;
        }
        __syncwarp();
        fill = 0;
      };
      for (int row = 0; row < 9; ++row) {
        const int oy = row % 3 - 1, oz = row / 3 - 1;
        const int jy = (cy + oy + nc) % nc, jz = (cz + oz + nc) % nc;
        const int64_t rb = R.cell0 + ((int64_t)jz * nc + jy) * nc;
        const bool contig = cx >= 1 && cx <= nc - 2;
        for (int piece = 0; piece < (contig ? 1 : 3); ++piece) {
          int ra, rbnd, b1, b2;
          if (contig) {  // cells cx-1, cx, cx+1 of the row are contiguous
            ra = d.cellstart[rb + cx - 1];
            rbnd = d.cellstart[rb + cx + 2];
            b1 = d.cellstart[rb + cx];
            b2 = d.cellstart[rb + cx + 1];
          } else {
            const int ox = piece - 1;
            const int jx = (cx + ox + nc) % nc;
            ra = d.cellstart[rb + jx];
            rbnd = d.cellstart[rb + jx + 1];
            b1 = ox == -1 ? rbnd : ra;  // every j of this cell gets offset ox
            b2 = ox == 1 ? ra : rbnd;
          }
          for (int jb = ra; jb < rbnd;) {
            const int take = min(rbnd - jb, kStageBatch - fill);
            if (lane < 32) {
              for (int u = lane; u < take; u += 32) {
                const int j = jb + u;
                const int ox = j < b1 ? -1 : (j < b2 ? 0 : 1);
                const V4 pj = Vec4<TF>::load(rel + j);
                V4 t;
                t.x = pj.x + ox * edge;
                t.y = pj.y + oy * edge;
                t.z = pj.z + oz * edge;
                t.w = TF(0);
                sxyz[wl][fill + u] = t;
                stag[wl][fill + u] = list_entry(j, ox, oy, oz);
              }
            }
            fill += take;
            jb += take;
            if (fill == kStageBatch) flush();
          }
        }
      }
      if (fill > 0) flush();
      s = e;
    }
    if (a0 + lane < a1 && rebuilds(d, d.rep_of_atom[a0 + lane])) d.nnb[a0 + lane] = list_count(d, cnt);
  }
}

// Verlet-list build, i-parallel: one warp per chunk of 32 consecutive atoms
// of the cell-sorted order, lane l owning atom a0 + l (the same list layout
// as k_build).  The chunk's lanes are taken in groups that share a replica
// and a cell row (y, z) -- one group for most chunks.  A group visits, row by
// row of its 9 neighbour rows, the x-cells from one left of its leftmost
// cell to one right of its rightmost (unwrapped, so a cell may come twice
// when the row is short; the second image is then at least one cell edge
// away and fails the distance test), every candidate j once for all lanes
// (one broadcast load), and each lane appends an accepted j to its own list
// column.  No ballot or shuffle per candidate; the entry order (row, then
// x-cell, then j) is the order k_build produces.
template <typename TF, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_build_ip(Sys d, LJ<TF> lj) {
  using V4 = typename Vec4<TF>::type;
  if (!any_rebuild(d)) return;
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int64_t n = d.n;
  const V4 *rel = static_cast<const V4 *>(d.rel);
  const int64_t nchunks = (n + 31) / 32;
  for (int64_t q = blockIdx.x * (int64_t)WARPS + wl; q < nchunks; q += (int64_t)gridDim.x * WARPS) {
    const int64_t i = q * 32 + lane;
    const bool act = i < n;
    int r = -1, cx = 0, cy = 0, cz = 0;
    V4 pi;
    pi.x = pi.y = pi.z = TF(0);
    if (act) {
      r = d.rep_of_atom[i];
      unpack_cell(d.cpk[i], cx, cy, cz);
      pi = Vec4<TF>::load(rel + i);
    }
    const bool mine = act && rebuilds(d, r);
    uint32_t *col = d.nbr + q * d.maxnb * 32 + lane;
    int cnt = 0;
    unsigned todo = __ballot_sync(0xffffffffu, mine);
    while (todo) {
      const int lead = __ffs(todo) - 1;
      const int gr = __shfl_sync(0xffffffffu, r, lead);
      const int gy = __shfl_sync(0xffffffffu, cy, lead);
      const int gz = __shfl_sync(0xffffffffu, cz, lead);
      const bool in = mine && r == gr && cy == gy && cz == gz;
      todo &= ~__ballot_sync(0xffffffffu, in);
      const int xlo = __reduce_min_sync(0xffffffffu, in ? cx : 0x7fffffff) - 1;
      const int xhi = -__reduce_min_sync(0xffffffffu, in ? -cx : 0x7fffffff) + 1;
      const Rep &R = d.rep[gr];
      const int nc = R.nc;
      const TF edge = (TF)R.edge;
      for (int row = 0; row < 9; ++row) {
        const int oy = row % 3 - 1, oz = row / 3 - 1;
        const int jy = (gy + oy + nc) % nc, jz = (gz + oz + nc) % nc;
        const int64_t rb = R.cell0 + ((int64_t)jz * nc + jy) * nc;
        const TF offy = oy * edge, offz = oz * edge;
        for (int ux = xlo; ux <= xhi; ++ux) {
          const int jx = (ux + nc) % nc;
          const int j0 = d.cellstart[rb + jx], j1 = d.cellstart[rb + jx + 1];
          const int ox = ux - cx;  // this lane's image offset (|ox| <= 1 for an accepted j)
          const TF offx = ox * edge;
          const int oxe = max(-1, min(1, ox));
          for (int j = j0; j < j1; ++j) {
            const V4 pj = Vec4<TF>::load(rel + j);
            V4 t;
            t.x = pj.x + offx;
            t.y = pj.y + offy;
            t.z = pj.z + offz;
            const TF dx = pi.x - t.x, dy = pi.y - t.y, dz = pi.z - t.z;
            const TF r2 = dx * dx + dy * dy + dz * dz;
            if (in && r2 < lj.rlist2 && (int64_t)j != i) {
              if (cnt < d.maxnb) col[(int64_t)cnt * 32] = list_entry(j, oxe, oy, oz);
              ++cnt;
            }
          }
        }
      }
    }
    if (mine) d.nnb[i] = list_count(d, cnt);
  }
}

}  // namespace
}  // namespace otf

using namespace otf;

// One tiling of the handle's replicas: tiles of at most ext[a] cells along
// each axis, its window capacity and CTA size.
struct TilePlan {
  int ext[3] = {3, 2, 2};
  std::vector<Tile> tiles;
  int wcap = 0;
  int threads = 0;
  double mean_tile = 0.0;
};

struct md_handle_s {
  md_params prm{};
  Sys d{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  // graphR[r]: r steps (1..kGraphSteps) in one graph, each step's correlator
  // pushes overlapping the next step; built on first use
  cudaGraphExec_t graphR[kGraphSteps + 1] = {};
  cudaStream_t side = nullptr;       // the correlator pushes run here, beside the next step
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_ring = nullptr;  // md_init: the velocity correlator's ring zeroed (side stream)
  bool vacf_pending = false;         // correlator pushes on `side` the next reduction must wait for
  // timed graphs (md_set_timing with graphs), each with its own event
  // records inside: sets 0 and 1 are two instances of the kGraphSteps-step
  // graph, replayed alternately so that one is read while the other runs;
  // set 1 + r holds the r-step graph (r < kGraphSteps) of a call's remainder
  static constexpr int kTimedSets = kGraphSteps + 1;
  cudaGraphExec_t graphT[kTimedSets] = {};
  std::vector<cudaEvent_t> tev[kTimedSets];
  std::vector<int> tev_class[kTimedSets];
  bool tev_pending[kTimedSets] = {};
  int tset = -1;                     // the set KTimer records into while capturing (-1: eager pool)
  bool fp64 = true;
  int nrep = 1;
  int red_blocks = 1;                // reduction CTAs over all replicas
  int pair_threads = kPairThreads;   // launch shapes (autotuned when asked)
  int build_warps = kCellWarps;
  int build_kind = 0;                // 0: j-parallel k_build, 1: i-parallel k_build_ip, 2: k_build_staged
  int tile_threads = 0;              // MD_PAIR_TILES: threads per tile CTA
  Tile *d_tiles = nullptr;
  std::vector<Rep> reps;             // host copy of the descriptor table
  Rep *d_rep = nullptr;
  int *d_rep_of_atom = nullptr, *d_rep_of_cell = nullptr, *d_rep_of_block = nullptr;
  double *d_lam = nullptr;
  int64_t steps_done = 0;
  int64_t corr_base = 0;
  corr_handle banks[kNBanks];  // system-owned correlators (borrowed by md_corr)
  bool bank_on[kNBanks] = {false, false, false, false};
  double *d_out = nullptr;  // unsort staging [16][n]
  char *arena = nullptr;    // one device allocation holding every per-atom, per-cell and per-tile array
  std::vector<Tile> tiles_host;  // MD_PAIR_TILES: the tile table in use
  std::vector<TilePlan> tile_plans;  // MD_PAIR_TILES: the candidate tilings ([0]: the default)
  int tile_plan = 0;                        // the one in use
  size_t tile_rec_cap = 0, tile_cell_cap = 0;  // per-tile array capacity (records, window-cell bytes)
  ObsDev *h_obs = nullptr;  // pinned [nrep]
  StepDev *h_st = nullptr;  // pinned
  unsigned *h_err = nullptr;
  double *h_lam = nullptr;  // pinned [nrep]
  // timing
  bool timing = false;
  std::vector<cudaEvent_t> ev;
  size_t ev_used = 0;
  std::vector<int> ev_class;
  double kms[MD_NKCLASS] = {0};
  int64_t klaunch[MD_NKCLASS] = {0};
  Spme spme;  // reciprocal-space Ewald (MD_POT_BUCK_EWALD)
};

namespace {

int grid_for(int64_t n, int threads, int max_blocks = 152 * 8) {
  return std::max(1, std::min(ceil_div(n, threads), max_blocks));
}

// Verlet lists (with the skin rule) in either list mode.
bool uses_lists(const md_params &p) { return p.pair_mode == MD_PAIR_VERLET || p.pair_mode == MD_PAIR_TILES; }

template <typename TF>
LJ<TF> lj_of(const md_params &p) {
  LJ<TF> lj;
  const double sr = p.sigma / p.rc;
  const double sr6 = sr * sr * sr * sr * sr * sr;
  const double s6 = p.sigma * p.sigma * p.sigma * p.sigma * p.sigma * p.sigma;
  lj.c12 = (TF)(4.0 * p.eps * s6 * s6);
  lj.c6 = (TF)(4.0 * p.eps * s6);
  lj.f12 = (TF)(48.0 * p.eps * s6 * s6);
  lj.f6 = (TF)(24.0 * p.eps * s6);
  lj.rc2 = (TF)(p.rc * p.rc);
  lj.ushift = (TF)(p.shift ? 4.0 * p.eps * (sr6 * sr6 - sr6) : 0.0);
  const double rl = p.rc + (uses_lists(p) ? p.skin : 0.0);
  lj.rlist2 = (TF)(rl * rl);
  // mixed-form Lennard-Jones: pairs closer than 1.03 sigma (|dF/dr| > 280
  // eps/sigma^2) get the displacement rounded once from the double-float
  // offsets; none in FP64 or for the ionic potential
  const double rclose = (std::is_same<TF, float>::value && p.potential == MD_POT_LJ) ? kRClose * p.sigma : 0.0;
  lj.rclose2 = (TF)(rclose * rclose);
  lj.rcb2 = (TF)((rclose + p.skin) * (rclose + p.skin));
  lj.A = (TF)p.buck_A;
  lj.inv_rho = (TF)(p.buck_rho > 0 ? 1.0 / p.buck_rho : 0.0);
  lj.C6 = (TF)p.buck_C;
  lj.alpha = (TF)p.ewald_alpha;
  lj.c2 = (TF)(2.0 * p.ewald_alpha / std::sqrt(3.14159265358979323846));
  lj.ke = (TF)p.coulomb;
  return lj;
}

// Event bracket around one kernel class when timing is on.
struct KTimer {
  md_handle *h;
  cudaStream_t s;
  int cls;
  KTimer(md_handle *h_, cudaStream_t s_, int cls_) : h(h_), s(s_), cls(cls_) { mark(); }
  ~KTimer() { mark(); }
  void mark() {
    if (!h || !h->timing) return;
    if (h->tset >= 0) {  // capturing a timed graph: an event-record node
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      h->tev[h->tset].push_back(e);
      h->tev_class[h->tset].push_back(cls);
      cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
      return;
    }
    if (h->ev_used == h->ev.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      h->ev.push_back(e);
      h->ev_class.push_back(cls);
    }
    h->ev_class[h->ev_used] = cls;
    cudaEventRecord(h->ev[h->ev_used++], s);
  }
};

template <typename TF>
void launch_build(const md_handle *h, cudaStream_t s) {
  const Sys &d = h->d;
  const int64_t chunks = (d.n + 31) / 32;
  const LJ<TF> lj = lj_of<TF>(h->prm);
  if (h->build_kind == 2) {
    if (h->build_warps == 8)
      k_build_staged<TF, 8><<<std::min(ceil_div(chunks, 8), 152 * 4), 256, 0, s>>>(d, lj);
    else
      k_build_staged<TF, 4><<<std::min(ceil_div(chunks, 4), 152 * 8), 128, 0, s>>>(d, lj);
    return;
  }
  if (h->build_kind == 1) {
    if (h->build_warps == 8)
      k_build_ip<TF, 8><<<std::min(ceil_div(chunks, 8), 152 * 8), 256, 0, s>>>(d, lj);
    else
      k_build_ip<TF, 4><<<std::min(ceil_div(chunks, 4), 152 * 16), 128, 0, s>>>(d, lj);
    return;
  }
  switch (h->build_warps) {
    case 2:
      k_build<TF, 2><<<std::min(ceil_div(chunks, 2), 152 * 16), 64, 0, s>>>(d, lj);
      break;
    case 8:
      k_build<TF, 8><<<std::min(ceil_div(chunks, 8), 152 * 8), 256, 0, s>>>(d, lj);
      break;
    default:
      k_build<TF, 4><<<std::min(ceil_div(chunks, 4), 152 * 16), 128, 0, s>>>(d, lj);
  }
}

template <typename TF>
int launch_rebuild(md_handle *h, cudaStream_t s) {
  const Sys &d = h->d;
  KTimer tm(h, s, MD_K_REBUILD);
  k_rb_zero<<<grid_for(d.ncell, kThreads), kThreads, 0, s>>>(d);
  if (h->fp64)
    k_rb_assign64<<<grid_for(d.n, kThreads), kThreads, 0, s>>>(d);
  else
    k_rb_assign_df<<<grid_for(d.n, kThreads), kThreads, 0, s>>>(d);
  k_rb_scan<<<1, 1024, 0, s>>>(d);
  k_rb_place<<<grid_for(d.n, kThreads), kThreads, 0, s>>>(d);
  k_rb_rank<TF><<<grid_for(d.ncell * 32, kCellWarps * 32), kCellWarps * 32, 0, s>>>(d);
  if (h->prm.pair_mode == MD_PAIR_VERLET) launch_build<TF>(h, s);
  if (h->prm.pair_mode == MD_PAIR_TILES)
    k_build_tile<<<d.ntiles, h->tile_threads, tile_smem(d.wcap, false), s>>>(d, lj_of<float>(h->prm));
  OTF_LAUNCH_CHECK();
  return MD_OK;
}

template <typename TF, int POT>
void launch_pair_pot(const md_handle *h, cudaStream_t s) {
  const Sys &d = h->d;
  if (h->prm.pair_mode == MD_PAIR_TILES) {
    if constexpr (std::is_same<TF, float>::value && POT == kPotLJ)
      k_pair_tile<<<d.ntiles, h->tile_threads, tile_smem(d.wcap, true), s>>>(
          d, lj_of<float>(h->prm));
  } else if (h->prm.pair_mode == MD_PAIR_VERLET) {
    if constexpr (std::is_same<TF, float>::value)
      k_pair_mixed<POT><<<ceil_div(d.n, h->pair_threads), h->pair_threads, 0, s>>>(d, lj_of<float>(h->prm));
    else
      k_pair_list<TF, POT><<<ceil_div(d.n, h->pair_threads), h->pair_threads, 0, s>>>(d, lj_of<TF>(h->prm));
  } else
    k_cells<TF, POT><<<std::min(ceil_div(d.ncell, kCellWarps), 152 * 16), kCellWarps * 32, 0, s>>>(
        d, lj_of<TF>(h->prm));
}

// Pair forces, then (MD_POT_BUCK_EWALD) the reciprocal-space Ewald terms
// added on top.
template <typename TF>
int launch_pair(md_handle *h, cudaStream_t s) {
  const Sys &d = h->d;
  {
    KTimer tm(h, s, MD_K_PAIR);
    if (h->prm.potential == MD_POT_BUCK_EWALD)
      launch_pair_pot<TF, kPotBuck>(h, s);
    else
      launch_pair_pot<TF, kPotLJ>(h, s);
    OTF_LAUNCH_CHECK();
  }
  if (h->spme.on()) {
    KTimer tm(h, s, MD_K_SPME);
    SpmeAtoms a;
    a.n = d.n;
    a.cpk = d.cpk;
    a.rel = d.rel;
    a.rlo = d.rlo;
    a.edge = h->reps[0].edge;
    a.cellstart = d.cellstart;
    a.nc = h->reps[0].nc;
    if (int rc = h->spme.run(a, d.F, d.epot, d.W, s)) return rc;
  }
  return MD_OK;
}

template <typename TF, typename A, bool KICK>
int launch_reduce(md_handle *h, cudaStream_t s) {
  KTimer tm(h, s, MD_K_REDUCE);
  k_kick_reduce<TF, A, KICK><<<h->red_blocks, kThreads, 0, s>>>(h->d, 0.5 * h->prm.dt);
  OTF_LAUNCH_CHECK();
  return MD_OK;
}

bool scalar_banks_on(const md_handle *h) { return h->bank_on[0] || h->bank_on[1] || h->bank_on[3]; }

// The waiting velocity-correlator pushes: a full block, or all of them when
// flushing.
int launch_vacf_block(md_handle *h, cudaStream_t s, bool flush) {
  const int block = std::min(kPushBlock, h->prm.vacf.p - h->prm.vacf.m + 1);  // see BlockIdx
  const BlockIdx bi{&h->d.st->step, &h->d.st->corr_base, h->prm.vacf.u, &h->d.st->vacf_done,
                    &h->d.st->vacf_ctas, std::max(block, 1), flush ? 1 : 0, h->d.err};
  return h->banks[2].c.launch_push_block(h->d.vbuf, !h->fp64, bi, s);
}

// The scalar correlator samples of the step just reduced (on s).
int launch_push_scalars(md_handle *h, cudaStream_t s) {
  KTimer tm(h, s, MD_K_REDUCE);
  CorrDev cs = h->bank_on[0] ? h->banks[0].c.dev : CorrDev{};
  CorrDev ch = h->bank_on[1] ? h->banks[1].c.dev : CorrDev{};
  CorrDev cm = h->bank_on[3] ? h->banks[3].c.dev : CorrDev{};
  const int64_t threads = (int64_t)h->nrep * 12;
  k_push_scalars<<<(int)ceil_div(threads, 128), 128, 0, s>>>(
      h->d, cs, h->bank_on[0] ? h->prm.stress.u : 0, ch, h->bank_on[1] ? h->prm.heatflux.u : 0, cm,
      h->bank_on[3] ? h->prm.massflux.u : 0);
  OTF_LAUNCH_CHECK();
  return MD_OK;
}

template <typename TF, typename A>
int launch_step(md_handle *h, cudaStream_t s, bool overlap) {
  const Sys &d = h->d;
  {
    KTimer tm(h, s, MD_K_INTEGRATE);
    if constexpr (std::is_same<TF, double>::value)
      k_kick_drift64<<<ceil_div(d.n, kThreads), kThreads, 0, s>>>(d, 0.5 * h->prm.dt);
    else
      k_kick_drift_df<<<ceil_div(d.n, kThreads), kThreads, 0, s>>>(d);
    OTF_LAUNCH_CHECK();
  }
  int rc = launch_rebuild<TF>(h, s);
  if (rc) return rc;
  if ((rc = launch_pair<TF>(h, s))) return rc;
  // the previous step's correlator pushes read the observables, the velocity
  // buffer and the step counter this reduction rewrites
  if (h->vacf_pending) {
    OTF_CUDA(cudaStreamWaitEvent(s, h->ev_join, 0));
    h->vacf_pending = false;
  }
  if ((rc = launch_reduce<TF, A, true>(h, s))) return rc;
  if (h->bank_on[2] || scalar_banks_on(h)) {
    // the pushes only read this step's observables and velocities, so they
    // can run beside the next step's integration, sort and forces (forked
    // onto `side`)
    cudaStream_t ps = overlap ? h->side : s;
    if (overlap) {
      OTF_CUDA(cudaEventRecord(h->ev_fork, s));
      OTF_CUDA(cudaStreamWaitEvent(ps, h->ev_fork, 0));
    }
    if (scalar_banks_on(h) && (rc = launch_push_scalars(h, ps))) return rc;
    if (h->bank_on[2]) {
      // the pushes wait in their input slots and are applied a block at a
      // time (the launches return at once until a block is full); one per
      // step for p > 16
      KTimer tm(h, ps, MD_K_VACF);
      if (h->d.vacf_slots > 1) {
        if ((rc = launch_vacf_block(h, ps, false))) return rc;
      } else {
        const PushIdx pi{&h->d.st->step, &h->d.st->corr_base, h->prm.vacf.u, 0};
        if ((rc = h->banks[2].c.launch_push(h->d.vbuf, h->d.vbuf, !h->fp64, pi, ps))) return rc;
      }
    }
    if (overlap) {
      OTF_CUDA(cudaEventRecord(h->ev_join, ps));
      h->vacf_pending = true;
    }
  }
  return MD_OK;
}

int step_once(md_handle *h, cudaStream_t s, bool overlap = false) {
  return h->fp64 ? launch_step<double, double>(h, s, overlap) : launch_step<float, float>(h, s, overlap);
}

// Waits (on s) for correlator pushes still running beside the step sequence.
int join_vacf(md_handle *h, cudaStream_t s) {
  if (!h->vacf_pending) return MD_OK;
  OTF_CUDA(cudaStreamWaitEvent(s, h->ev_join, 0));
  h->vacf_pending = false;
  return MD_OK;
}

int refresh_obs(md_handle *h) {
  return h->fp64 ? launch_reduce<double, double, false>(h, h->stream)
                 : launch_reduce<float, float, false>(h, h->stream);
}

int check_device(md_handle *h) {
  OTF_CUDA(cudaMemcpyAsync(h->h_err, h->d.err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  OTF_CUDA(cudaStreamSynchronize(h->stream));
  const unsigned e = *h->h_err;
  if (e) {
    set_error("device check failed (flags 0x%x):%s%s%s%s%s", e, (e & ERR_NONFINITE) ? " non-finite coordinates;" : "",
              (e & ERR_NBR_OVERFLOW) ? " neighbour list over capacity (raise max_neighbors);" : "",
              (e & ERR_BAD_TYPE) ? " atom type out of range;" : "",
              (e & ERR_PUSH_BACKLOG) ? " velocity-correlator pushes left unapplied;" : "",
              (e & ERR_WINDOW) ? " a tile window outgrew its shared-memory capacity (use MD_PAIR_VERLET);" : "");
    return MD_ESTATE;
  }
  return MD_OK;
}

// Captures `steps` steps into one graph; with several, each velocity push
// overlaps the next step (the graph ends joined).
int capture_steps(md_handle *h, int steps, cudaGraphExec_t *out) {
  cudaGraph_t g = nullptr;
  OTF_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = MD_OK;
  for (int k = 0; k < steps && !rc; ++k) rc = step_once(h, h->cap_stream, steps > 1);
  if (!rc) rc = join_vacf(h, h->cap_stream);
  h->vacf_pending = false;
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) {
    set_error("graph capture failed: %s", cudaGetErrorString(e));
    return MD_ECUDA;
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *out = nullptr;
    set_error("graph instantiate failed: %s", cudaGetErrorString(e));
    return MD_ECUDA;
  }
  return MD_OK;
}

// The r-step graph (captured on first use).
int graph_of(md_handle *h, int r, cudaGraphExec_t *out) {
  if (!h->graphR[r]) {
    const int rc = capture_steps(h, r, &h->graphR[r]);
    if (rc) return rc;
  }
  *out = h->graphR[r];
  return MD_OK;
}

// Timed graph set k (see md_handle::graphT), captured on first use.
int timed_graph_of(md_handle *h, int k, cudaGraphExec_t *out) {
  if (!h->graphT[k]) {
    h->tset = k;
    const int rc = capture_steps(h, k < 2 ? kGraphSteps : k - 1, &h->graphT[k]);
    h->tset = -1;
    if (rc) return rc;
  }
  *out = h->graphT[k];
  return MD_OK;
}

int launch_graph(cudaGraphExec_t g, cudaStream_t s) {
  const cudaError_t e = cudaGraphLaunch(g, s);
  if (e != cudaSuccess) {
    set_error("cudaGraphLaunch failed: %s", cudaGetErrorString(e));
    return MD_ECUDA;
  }
  return MD_OK;
}

// The velocity pushes still waiting in their input slots (fewer than a
// block), applied on the system's stream.  Runs before every readout of the
// velocity correlator, so a read always sees every step taken, while md_step
// itself leaves a partial block waiting for the next call.
int flush_vacf(void *ctx) {
  md_handle *h = static_cast<md_handle *>(ctx);
  if (!h->bank_on[2] || h->d.vacf_slots <= 1) return MD_OK;
  return launch_vacf_block(h, h->stream, true);
}

// Waits for the last replay of timed graph k and adds its kernel times to
// the counters (its events come in start / stop pairs).
int read_timed(md_handle *h, int k) {
  if (!h->tev_pending[k]) return MD_OK;
  h->tev_pending[k] = false;
  const std::vector<cudaEvent_t> &ev = h->tev[k];
  for (size_t e = 0; e + 1 < ev.size(); e += 2) {
    OTF_CUDA(cudaEventSynchronize(ev[e + 1]));
    float ms = 0.f;
    OTF_CUDA(cudaEventElapsedTime(&ms, ev[e], ev[e + 1]));
    h->kms[h->tev_class[k][e]] += ms;
    h->klaunch[h->tev_class[k][e]] += 1;
  }
  return MD_OK;
}

int validate_params(const md_params *p) {
  if (!p) {
    set_error("md_init: null parameters");
    return MD_EINVAL;
  }
  if (!(p->rc > 0) || !(p->sigma > 0) || !(p->dt > 0) || p->skin < 0 || !std::isfinite(p->eps)) {
    set_error("md_init: rc, sigma, dt must be positive and skin >= 0");
    return MD_EINVAL;
  }
  if (p->ntypes < 1 || p->ntypes > 8) {
    set_error("md_init: ntypes must be in [1, 8]");
    return MD_EINVAL;
  }
  for (int t = 0; t < p->ntypes; ++t)
    if (!(p->mass[t] > 0)) {
      set_error("md_init: mass[%d] must be positive", t);
      return MD_EINVAL;
    }
  if (p->precision != MD_PREC_FP64 && p->precision != MD_PREC_MIXED) {
    set_error("md_init: unknown precision");
    return MD_EINVAL;
  }
  if (p->list_build < 0 || p->list_build > 3) {
    set_error("md_init: list_build must be 0, 1, 2 or 3");
    return MD_EINVAL;
  }
  if (p->pair_mode != MD_PAIR_VERLET && p->pair_mode != MD_PAIR_CELLS && p->pair_mode != MD_PAIR_TILES) {
    set_error("md_init: unknown pair_mode");
    return MD_EINVAL;
  }
  if (p->window_slots < 0 || p->window_slots > kWinMaxSlots || (p->window_slots > 0 && p->window_slots % 16)) {
    set_error("md_init: window_slots must be 0 (automatic) or a multiple of 16 up to 4096");
    return MD_EINVAL;
  }
  if (p->pair_mode == MD_PAIR_TILES && (p->precision != MD_PREC_MIXED || p->potential != MD_POT_LJ)) {
    set_error("md_init: MD_PAIR_TILES is for the mixed-precision Lennard-Jones form");
    return MD_EINVAL;
  }
  if (p->potential == MD_POT_BUCK_EWALD) {
    if (!(p->buck_A >= 0) || !(p->buck_rho > 0) || !(p->buck_C >= 0) || !(p->coulomb > 0) ||
        !(p->ewald_alpha > 0)) {
      set_error("md_init: Buckingham-Ewald needs A >= 0, rho > 0, C >= 0, coulomb > 0, ewald_alpha > 0");
      return MD_EINVAL;
    }
    if ((p->order != 4 && p->order != 6 && p->order != 8) || p->mesh < p->order || p->mesh % 2 || p->mesh > 512) {
      set_error("md_init: SPME needs order 4, 6 or 8 and an even mesh in [order, 512]");
      return MD_EINVAL;
    }
    for (int t = 0; t < p->ntypes; ++t)
      if (!std::isfinite(p->charge[t])) {
        set_error("md_init: charge[%d] is not finite", t);
        return MD_EINVAL;
      }
  } else if (p->potential != MD_POT_LJ) {
    set_error("md_init: unknown potential");
    return MD_EINVAL;
  }
  if (p->flux_species < 0 || p->flux_species >= p->ntypes) {
    set_error("md_init: flux_species must be a type in [0, ntypes)");
    return MD_EINVAL;
  }
  const corr_spec *cs[kNBanks] = {&p->stress, &p->heatflux, &p->vacf, &p->massflux};
  for (int k = 0; k < kNBanks; ++k) {
    if (cs[k]->u < 0) {
      set_error("md_init: correlator update interval must be >= 0");
      return MD_EINVAL;
    }
    if (cs[k]->u == 0) continue;
    corr_params cp{cs[k]->b, cs[k]->p, cs[k]->m, 0, 3, 1, MD_PREC_FP64, 1.0};
    if (validate_corr_params(cp)) return MD_EINVAL;
  }
  return MD_OK;
}

int validate_replicas(const md_params *p, const md_replica *reps, int count, int mem) {
  if (!reps || count < 1) {
    set_error("md_init: at least one replica is needed");
    return MD_EINVAL;
  }
  if (mem != MD_MEM_HOST && mem != MD_MEM_DEVICE) {
    set_error("md_init: mem must be MD_MEM_HOST or MD_MEM_DEVICE");
    return MD_EINVAL;
  }
  if (p->potential == MD_POT_BUCK_EWALD && count > 1) {
    set_error("md_init: the Buckingham-Ewald potential is for a single system");
    return MD_EINVAL;
  }
  if (p->potential == MD_POT_BUCK_EWALD && !(2.0 * p->rc < reps[0].box)) {
    set_error("md_init: the real-space cutoff must be below half the box");
    return MD_EINVAL;
  }
  if (count > 1 && p->vacf.u > 0) {
    set_error("md_init: the per-atom velocity correlator is for a single system (set vacf.u = 0)");
    return MD_EINVAL;
  }
  const double rl = p->rc + (uses_lists(*p) ? p->skin : 0.0);
  int64_t total = 0;
  for (int k = 0; k < count; ++k) {
    const md_replica &R = reps[k];
    if (R.n < 2 || (count > 1 && R.n < kMaxPairThreads)) {
      set_error("md_init: replica %d has %lld atoms (at least %d per replica when there are several)", k,
                (long long)R.n, count > 1 ? kMaxPairThreads : 2);
      return MD_EINVAL;
    }
    if (!(R.box > 0) || !R.r || !R.v) {
      set_error("md_init: replica %d needs a positive box and r, v arrays", k);
      return MD_EINVAL;
    }
    const int nc = (int)std::floor(R.box / rl);
    if (nc < 3) {
      set_error("md_init: replica %d: box %.6g holds fewer than 3 cells of edge rc + skin = %.6g", k, R.box, rl);
      return MD_EINVAL;
    }
    if (nc > 1023) {
      set_error("md_init: replica %d has more than 1023 cells per side", k);
      return MD_EINVAL;
    }
    total += R.n;
    // the values themselves (finite coordinates and velocities, types in
    // range) are checked on the device after the copy, for host and device
    // arrays alike (k_check_finite, and the first sort for the types)
  }
  if (total >= (int64_t(1) << 26)) {  // 26 bits of atom index per neighbour-list entry
    set_error("md_init: %lld atoms in total; at most 2^26 - 1", (long long)total);
    return MD_EINVAL;
  }
  return MD_OK;
}

void release(md_handle *h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (cudaGraphExec_t g : h->graphR)
    if (g) cudaGraphExecDestroy(g);
  for (int k = 0; k < md_handle::kTimedSets; ++k) {
    if (h->graphT[k]) cudaGraphExecDestroy(h->graphT[k]);
    for (cudaEvent_t e : h->tev[k]) cudaEventDestroy(e);
  }
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->side) {
    cudaStreamSynchronize(h->side);
    cudaStreamDestroy(h->side);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_ring) cudaEventDestroy(h->ev_ring);
  // every device array of the handle lives in the arena, except the
  // particles' readout staging
  if (h->arena) cudaFree(h->arena);
  if (h->d_out) cudaFree(h->d_out);
  h->spme.destroy();
  for (int k = 0; k < kNBanks; ++k)
    if (h->bank_on[k]) h->banks[k].c.destroy();
  if (h->h_obs) cudaFreeHost(h->h_obs);
  if (h->h_st) cudaFreeHost(h->h_st);
  if (h->h_err) cudaFreeHost(h->h_err);
  if (h->h_lam) cudaFreeHost(h->h_lam);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  delete h;
}

// Device time of `reps` runs of fn on the handle's stream (ms per run).
template <typename Fn>
float time_runs(md_handle *h, int reps, Fn fn) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  fn();  // warm
  cudaEventRecord(a, h->stream);
  for (int k = 0; k < reps; ++k) fn();
  cudaEventRecord(b, h->stream);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / reps;
}

// Autotuner: times the pair kernel at 64 / 128 / 256 threads per CTA and
// the list build (j-parallel at 2 / 4 / 8 warps per CTA, i-parallel and staged at 4 / 8)
// on the system itself (forces
// and lists are recomputed from the unchanged state, so the trajectory is
// not touched) and keeps the fastest of each.
int autotune_tiles(md_handle *h);

template <typename TF>
int autotune(md_handle *h) {
  if (h->prm.pair_mode == MD_PAIR_TILES) return autotune_tiles(h);
  if (h->prm.pair_mode != MD_PAIR_VERLET) return MD_OK;  // nothing to choose for the cell sweep
  float best = 1e30f;
  int best_t = h->pair_threads;
  for (int t : {64, 128, 256}) {
    h->pair_threads = t;
    const float ms = time_runs(h, 5, [&] { launch_pair<TF>(h, h->stream); });
    if (ms < best) best = ms, best_t = t;
  }
  h->pair_threads = best_t;
  best = 1e30f;
  int best_w = h->build_warps, best_k = h->build_kind;
  const int shapes[7][2] = {{0, 2}, {0, 4}, {0, 8}, {1, 4}, {1, 8}, {2, 4}, {2, 8}};
  for (const auto &kw : shapes) {
    h->build_kind = kw[0];
    h->build_warps = kw[1];
    const float ms = time_runs(h, 3, [&] {
      cudaMemsetAsync(h->d.rebuild, 1, (h->nrep + 1) * sizeof(int), h->stream);
      launch_build<TF>(h, h->stream);
    });
    if (ms < best) best = ms, best_w = kw[1], best_k = kw[0];
  }
  h->build_warps = best_w;
  h->build_kind = best_k;
  // rebuild the lists once more with the chosen shape, then the forces
  OTF_CUDA(cudaMemsetAsync(h->d.rebuild, 1, (h->nrep + 1) * sizeof(int), h->stream));
  launch_build<TF>(h, h->stream);
  OTF_LAUNCH_CHECK();
  if (int rc = launch_pair<TF>(h, h->stream)) return rc;
  OTF_CUDA(cudaMemsetAsync(h->d.rebuild, 0, (h->nrep + 1) * sizeof(int), h->stream));
  OTF_CUDA(cudaStreamSynchronize(h->stream));
  return MD_OK;
}

// Segments [start, start + len) of nearly equal length <= b covering 0..nc-1.
std::vector<std::pair<int, int>> tile_segments(int nc, int b) {
  const int nseg = (nc + b - 1) / b, base = nc / nseg, extra = nc % nseg;
  std::vector<std::pair<int, int>> out;
  for (int k = 0, x = 0; k < nseg; ++k) {
    const int len = base + (k < extra ? 1 : 0);
    out.emplace_back(x, len);
    x += len;
  }
  return out;
}

// MD_PAIR_TILES: the tile table, the window capacity (the largest window
// expected at 1.2 times a replica's mean density, or at least one atom per
// sigma^3, plus 64 slots), the CTA size (1.1 times the largest mean tile,
// 128..384 threads; the rare larger tile takes a second pass) and the list
// arrays.
// Threads per tile CTA: f times the largest mean tile, in warps, 128..384.
int tile_threads_for(double mean_tile, double f) {
  return std::max(128, std::min(kTileThreadsMax, ((int)std::ceil(f * mean_tile) + 31) / 32 * 32));
}

// Makes candidate tiling k, at `threads` per tile CTA, the handle's tiling
// (host side; finish_tiles uploads it).
void use_plan_host(md_handle *h, int k, int threads) {
  const TilePlan &tp = h->tile_plans[k];
  h->tile_plan = k;
  h->tiles_host = tp.tiles;
  h->d.ntiles = (int)tp.tiles.size();
  h->d.wcap = tp.wcap;
  h->tile_threads = threads;
}

int plan_tiles(const md_handle *h, const md_replica *reps, int count, const int ext[3], TilePlan &out) {
  const md_params &p = h->prm;
  out = TilePlan{};
  for (int a = 0; a < 3; ++a) out.ext[a] = ext[a];
  double need = 0.0, mean_win = 0.0, mean_tile = 0.0;
  for (int k = 0; k < count; ++k) {
    const Rep &R = h->reps[k];
    const auto sx = tile_segments(R.nc, ext[0]), sy = tile_segments(R.nc, ext[1]), sz = tile_segments(R.nc, ext[2]);
    int mx = 0, my = 0, mz = 0;
    for (const auto &z : sz)
      for (const auto &y : sy)
        for (const auto &x : sx) {
          Tile t{};
          t.rep = k;
          t.x0 = (unsigned short)x.first;
          t.y0 = (unsigned short)y.first;
          t.z0 = (unsigned short)z.first;
          t.bx = (unsigned char)x.second;
          t.by = (unsigned char)y.second;
          t.bz = (unsigned char)z.second;
          out.tiles.push_back(t);
          mx = std::max(mx, x.second);
          my = std::max(my, y.second);
          mz = std::max(mz, z.second);
        }
    const double cell_vol = R.edge * R.edge * R.edge;
    const double apc = reps[k].n / ((double)R.nc * R.nc * R.nc);
    const double s3 = p.sigma * p.sigma * p.sigma;
    const double win_cells = (double)(mx + 2) * (my + 2) * (mz + 2);
    need = std::max(need, win_cells * std::max(1.2 * apc, cell_vol / s3) + 64.0);
    mean_win = std::max(mean_win, win_cells * apc + 1.0);
    mean_tile = std::max(mean_tile, (double)mx * my * mz * apc);
  }
  out.wcap = std::min(kWinMaxSlots, ((int)std::ceil(need) + 63) / 64 * 64);
  if (p.window_slots > 0) out.wcap = p.window_slots;  // the caller's capacity (checked at every build)
  if ((p.window_slots == 0 && 1.1 * mean_win > out.wcap) || h->d.maxnb > 65528) {
    set_error("md_init: MD_PAIR_TILES: cells hold too many atoms for a shared-memory window "
              "(mean window %.0f slots of %d); use MD_PAIR_VERLET",
              mean_win, out.wcap);
    return MD_EINVAL;
  }
  out.mean_tile = mean_tile;
  out.threads = tile_threads_for(mean_tile, 1.1);
  return MD_OK;
}

// MD_PAIR_TILES: the tile table of tiles of at most 3 x 2 x 2 cells, the
// window capacity (the largest window expected at 1.2 times a replica's
// mean density, or at least one atom per sigma^3, plus 64 slots) and the
// CTA size (1.1 times the largest mean tile, 128..384 threads; the rare
// larger tile takes a second pass).  With md_params.autotune the other
// candidate tilings (2 x 2 x 2 and 3 x 3 x 2 cells) are planned too, and
// the per-tile arrays are sized for the largest of them.
int setup_tiles(md_handle *h, const md_replica *reps, int count) {
  static const int kExts[3][3] = {{3, 2, 2}, {2, 2, 2}, {3, 3, 2}};
  h->tile_plans.clear();
  for (int c = 0; c < (h->prm.autotune ? 3 : 1); ++c) {
    TilePlan tp;
    const int rc = plan_tiles(h, reps, count, kExts[c], tp);
    if (rc && c == 0) return rc;  // the default tiling must fit
    if (!rc) h->tile_plans.push_back(std::move(tp));
  }
  clear_error();
  h->tile_rec_cap = 0;
  h->tile_cell_cap = 0;
  for (const TilePlan &tp : h->tile_plans) {
    h->tile_rec_cap = std::max(h->tile_rec_cap, tp.tiles.size());
    h->tile_cell_cap = std::max(h->tile_cell_cap, tp.tiles.size() * (size_t)(tp.wcap + kWinPad));
  }
  use_plan_host(h, 0, h->tile_plans[0].threads);
  return MD_OK;
}

// MD_PAIR_TILES, once the arrays are carved (and again for every tiling the
// autotuner tries): the tile table uploaded, every record marked "no window"
// (natoms = -1) until the next list build, and the kernels' shared-memory
// limits set to the window size.
int finish_tiles(md_handle *h, cudaStream_t st) {
  Sys &d = h->d;
  const size_t nt = h->tiles_host.size();
  OTF_CUDA(cudaMemcpyAsync(h->d_tiles, h->tiles_host.data(), nt * sizeof(Tile), cudaMemcpyHostToDevice, st));
  OTF_CUDA(cudaMemsetAsync(d.trec, 0xff, nt * sizeof(TileWin), st));
  OTF_CUDA(cudaFuncSetAttribute(k_build_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tile_smem(d.wcap, false)));
  OTF_CUDA(cudaFuncSetAttribute(k_pair_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tile_smem(d.wcap, true)));
  return MD_OK;
}

// MD_PAIR_TILES autotuner (md_params.autotune): every candidate tiling
// whose windows fit (tiles of at most 3 x 2 x 2, 2 x 2 x 2 and 3 x 3 x 2
// cells) at 1.0, 1.1 and 1.3 times its largest mean tile in threads per
// CTA, timed on the system itself as one pair-kernel launch plus an eighth
// of a list build (a rebuild's share of a step at a skin of 0.3-0.4 sigma).
// A tiling whose build finds a window over capacity is dropped.  The
// fastest is kept, and the lists, window records and forces are rebuilt
// with it; the trajectory is not touched.
int autotune_tiles(md_handle *h) {
  const LJ<float> lj = lj_of<float>(h->prm);
  const size_t nflags = (size_t)(h->nrep + 1) * sizeof(int);
  auto build = [&] {
    cudaMemsetAsync(h->d.rebuild, 1, nflags, h->stream);
    k_build_tile<<<h->d.ntiles, h->tile_threads, tile_smem(h->d.wcap, false), h->stream>>>(h->d, lj);
  };
  float best = 1e30f;
  int best_k = 0, best_t = h->tile_threads;
  for (int k = 0; k < (int)h->tile_plans.size(); ++k) {
    int tried[3], ntried = 0;
    for (double f : {1.0, 1.1, 1.3}) {
      const int t = tile_threads_for(h->tile_plans[k].mean_tile, f);
      bool seen = false;
      for (int q = 0; q < ntried; ++q) seen = seen || tried[q] == t;
      if (seen) continue;
      tried[ntried++] = t;
      use_plan_host(h, k, t);
      if (int rc = finish_tiles(h, h->stream)) return rc;
      const float mb = time_runs(h, 2, build);
      OTF_LAUNCH_CHECK();
      OTF_CUDA(cudaMemcpyAsync(h->h_err, h->d.err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
      OTF_CUDA(cudaStreamSynchronize(h->stream));
      if (*h->h_err) {  // a window over capacity: not a candidate
        OTF_CUDA(cudaMemsetAsync(h->d.err, 0, sizeof(unsigned), h->stream));
        continue;
      }
      const float mp = time_runs(h, 5, [&] { launch_pair<float>(h, h->stream); });
      OTF_LAUNCH_CHECK();
      const float cost = mp + 0.125f * mb;
      if (cost < best) best = cost, best_k = k, best_t = t;
    }
  }
  use_plan_host(h, best_k, best_t);
  if (int rc = finish_tiles(h, h->stream)) return rc;
  build();
  OTF_LAUNCH_CHECK();
  if (int rc = launch_pair<float>(h, h->stream)) return rc;
  OTF_CUDA(cudaMemsetAsync(h->d.rebuild, 0, nflags, h->stream));
  OTF_CUDA(cudaStreamSynchronize(h->stream));
  return MD_OK;
}

// Device arrays carved out of one allocation: a driver allocation costs tens
// of microseconds whatever its size, and a handle has ~35 arrays.  The same
// sequence of take() calls runs twice: without a base to add up the sizes,
// then with the allocation to hand out the pointers (256-byte aligned).
struct Arena {
  char *base = nullptr;
  size_t used = 0;
  template <typename T>
  void take(T *&p, size_t bytes) {
    const size_t off = (used + 255) & ~size_t(255);
    used = off + bytes;
    p = base ? reinterpret_cast<T *>(base + off) : nullptr;
  }
};

int init_impl(md_handle *h, const md_params *p, const md_replica *reps, int count, int mem) {
  h->prm = *p;
  h->build_kind = p->list_build == 0 ? kDefaultBuildKind : p->list_build - 1;
  h->fp64 = p->precision == MD_PREC_FP64;
  h->nrep = count;
  Sys &d = h->d;
  const double rl = p->rc + (uses_lists(*p) ? p->skin : 0.0);
  // replica table: atoms, cells and reduction CTAs laid end to end
  h->reps.resize(count);
  int64_t n = 0, ncell = 0, blocks = 0;
  double rho_max = 0.0;
  for (int k = 0; k < count; ++k) {
    Rep &R = h->reps[k];
    R.nc = (int)std::floor(reps[k].box / rl);
    R.L = reps[k].box;
    R.edge = R.L / R.nc;
    const dfloat ef = df_from_double(R.edge);
    R.edge_h = ef.h;
    R.edge_l = ef.l;
    R.atom0 = n;
    R.atom1 = n + reps[k].n;
    R.cell0 = ncell;
    R.block0 = blocks;
    const int64_t per_cta = h->fp64 ? 4096 : kRedAtomsMixed;
    R.nblk = (int)std::max<int64_t>(1, std::min<int64_t>(kMaxRedBlocks, (reps[k].n + per_cta - 1) / per_cta));
    n += reps[k].n;
    ncell += (int64_t)R.nc * R.nc * R.nc;
    blocks += R.nblk;
    rho_max = std::max(rho_max, reps[k].n / (R.L * R.L * R.L));
  }
  d.n = n;
  d.ncell = ncell;
  d.nrep = count;
  h->red_blocks = (int)blocks;
  d.dt = p->dt;
  const double half_skin = 0.5 * (uses_lists(*p) ? p->skin : 0.0);
  d.lim2 = half_skin * half_skin;
  d.always_rebuild = (p->pair_mode == MD_PAIR_CELLS || p->skin <= 0.0) ? 1 : 0;
  d.ntypes = p->ntypes;
  for (int t = 0; t < 8; ++t) {
    d.mass[t] = t < p->ntypes ? p->mass[t] : 1.0;
    d.invm[t] = 1.0 / d.mass[t];
    d.charge[t] = (p->potential == MD_POT_BUCK_EWALD && t < p->ntypes) ? p->charge[t] : 0.0;
  }
  d.flux_species = p->flux_species;
  int maxnb = p->max_neighbors;
  if (maxnb <= 0) {
    const double mean = rho_max * 4.18879020478639 * rl * rl * rl;
    maxnb = ((int)(1.35 * mean + 24.0) + 7) / 8 * 8;
  }
  d.maxnb = maxnb;
  d.vacf_u = p->vacf.u;
  // blocked velocity pushes keep the p - 1 <= 15 most recent samples in
  // registers; no input slot at all when the velocity correlator is off
  d.vacf_slots = p->vacf.u <= 0 ? 0 : (p->vacf.p <= 16 ? kPushBlock : 1);
  d.maxchunks = (n + 31) / 32;  // 32-atom chunks of the neighbour lists
  d.unit_mass = 1;
  for (int t = 0; t < 8; ++t) {
    const dfloat hh = df_from_double(0.5 * p->dt * d.invm[t]);
    d.hdtm_h[t] = hh.h;
    d.hdtm_l[t] = hh.l;
    const dfloat mm = df_from_double(d.mass[t]);
    d.mass_h[t] = mm.h;
    d.mass_l[t] = mm.l;
    if (t < d.ntypes && d.mass[t] != 1.0) d.unit_mass = 0;
  }
  {
    const dfloat dtf = df_from_double(p->dt);
    d.dt_h = dtf.h;
    d.dt_l = dtf.l;
  }
  const size_t tf = h->fp64 ? sizeof(double) : sizeof(float);
  const size_t v4 = h->fp64 ? sizeof(dvec4) : sizeof(float4);
  OTF_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  OTF_CUDA(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
  OTF_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  OTF_CUDA(cudaEventCreateWithFlags(&h->ev_ring, cudaEventDisableTiming));
  OTF_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  if (p->pair_mode == MD_PAIR_TILES)
    if (int rc = setup_tiles(h, reps, count)) return rc;
  auto carve = [&](Arena &A) {
    if (h->fp64) {
      A.take(d.r, 3 * n * sizeof(double));
      A.take(d.v, 3 * n * sizeof(double));
    } else {
      A.take(d.rlo, n * sizeof(float4));
      A.take(d.vh, 3 * n * sizeof(float));
      A.take(d.vl, 3 * n * sizeof(float));
    }
    A.take(d.F, 3 * n * tf);
    A.take(d.epot, n * tf);
    A.take(d.W, 6 * n * tf);
    A.take(d.rel, n * v4);
    A.take(d.relb, n * v4);
    if (d.vacf_slots > 0) A.take(d.vbuf, (size_t)d.vacf_slots * 3 * n * tf);
    A.take(d.id, n * sizeof(int));
    A.take(d.type, n * sizeof(int));
    A.take(d.cpk, n * sizeof(int));
    A.take(d.rB, 3 * n * sizeof(double));
    A.take(d.vB, 3 * n * sizeof(double));
    A.take(d.idB, n * sizeof(int));
    A.take(d.typeB, n * sizeof(int));
    A.take(d.cellB, n * sizeof(int));
    A.take(d.slot, n * sizeof(int));
    A.take(d.perm, n * sizeof(int));
    A.take(d.cellcount, ncell * sizeof(int));
    A.take(d.cellstart, (ncell + 1) * sizeof(int));
    if (p->pair_mode == MD_PAIR_VERLET) A.take(d.nbr, (size_t)d.maxchunks * maxnb * 32 * sizeof(uint32_t));
    if (p->pair_mode == MD_PAIR_TILES) {
      A.take(h->d_tiles, h->tile_rec_cap * sizeof(Tile));
      A.take(d.tnb, (size_t)(d.maxnb / 8) * n * sizeof(uint4));
      A.take(d.tcl, (size_t)(kMaxCloseT / 8) * n * sizeof(uint4));
      A.take(d.trec, h->tile_rec_cap * sizeof(TileWin));
      A.take(d.tcell, h->tile_cell_cap);
    }
    A.take(d.nnb, n * sizeof(int));
    A.take(d.partials, (size_t)blocks * kNRed * sizeof(double));
    A.take(d.counter, count * sizeof(unsigned));
    A.take(d.obs, count * sizeof(ObsDev));
    A.take(d.st, sizeof(StepDev));
    A.take(d.rebuild, (count + 1) * sizeof(int));
    A.take(d.err, sizeof(unsigned));
    A.take(h->d_rep, count * sizeof(Rep));
    A.take(h->d_rep_of_atom, n * sizeof(int));
    A.take(h->d_rep_of_cell, ncell * sizeof(int));
    A.take(h->d_rep_of_block, blocks * sizeof(int));
    A.take(h->d_lam, count * sizeof(double));
  };
  {
    Arena sizes;
    carve(sizes);
    OTF_CUDA(cudaMalloc(&h->arena, sizes.used));
    Arena a;
    a.base = h->arena;
    carve(a);
  }
  d.tiles = h->d_tiles;
  OTF_CUDA(cudaMallocHost(&h->h_obs, count * sizeof(ObsDev)));
  OTF_CUDA(cudaMallocHost(&h->h_st, sizeof(StepDev)));
  OTF_CUDA(cudaMallocHost(&h->h_err, sizeof(unsigned)));
  OTF_CUDA(cudaMallocHost(&h->h_lam, count * sizeof(double)));
  d.rep = h->d_rep;
  d.rep_of_atom = h->d_rep_of_atom;
  d.rep_of_cell = h->d_rep_of_cell;
  d.rep_of_block = h->d_rep_of_block;
  d.lam = h->d_lam;
  cudaStream_t st = h->stream;
  if (p->pair_mode == MD_PAIR_TILES)
    if (int rc = finish_tiles(h, st)) return rc;
  // replica lookup tables (set-up only), filled on the device from the
  // descriptor table
  OTF_CUDA(cudaMemcpyAsync(h->d_rep, h->reps.data(), count * sizeof(Rep), cudaMemcpyHostToDevice, st));
  k_rep_of<<<grid_for(n, kThreads), kThreads, 0, st>>>(h->d_rep, count, 0, h->d_rep_of_atom, n);
  k_rep_of<<<grid_for(ncell, kThreads), kThreads, 0, st>>>(h->d_rep, count, 1, h->d_rep_of_cell, ncell);
  k_rep_of<<<grid_for(blocks, kThreads), kThreads, 0, st>>>(h->d_rep, count, 2, h->d_rep_of_block, blocks);
  OTF_LAUNCH_CHECK();
  OTF_CUDA(cudaMemsetAsync(d.counter, 0, count * sizeof(unsigned), st));
  OTF_CUDA(cudaMemsetAsync(d.obs, 0, count * sizeof(ObsDev), st));
  OTF_CUDA(cudaMemsetAsync(d.st, 0, sizeof(StepDev), st));
  OTF_CUDA(cudaMemsetAsync(d.err, 0, sizeof(unsigned), st));
  OTF_CUDA(cudaMemsetAsync(d.F, 0, 3 * n * tf, st));
  if (d.vacf_slots > 0) OTF_CUDA(cudaMemsetAsync(d.vbuf, 0, (size_t)d.vacf_slots * 3 * n * tf, st));
  OTF_CUDA(cudaMemsetAsync(d.rebuild, 1, (count + 1) * sizeof(int), st));  // every flag set (nonzero)
  // inputs, replica after replica, component-major within the whole system:
  // FP64 form straight into the state; mixed form through the scratch,
  // converted to cell + double-float offset by k_init_df below
  const cudaMemcpyKind kind = mem == MD_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  double *rdst = h->fp64 ? d.r : d.rB, *vdst = h->fp64 ? d.v : d.vB;
  for (int k = 0; k < count; ++k) {
    const Rep &R = h->reps[k];
    const int64_t nk = reps[k].n;
    for (int a = 0; a < 3; ++a) {
      OTF_CUDA(cudaMemcpyAsync(rdst + a * n + R.atom0, reps[k].r + a * nk, nk * sizeof(double), kind, st));
      OTF_CUDA(cudaMemcpyAsync(vdst + a * n + R.atom0, reps[k].v + a * nk, nk * sizeof(double), kind, st));
    }
    if (reps[k].type)
      OTF_CUDA(cudaMemcpyAsync(d.type + R.atom0, reps[k].type, nk * sizeof(int), kind, st));
    else
      OTF_CUDA(cudaMemsetAsync(d.type + R.atom0, 0, nk * sizeof(int), st));
  }
  // rdst and vdst hold 3n values each (FP64 state or the mixed form's scratch)
  k_check_finite<<<grid_for(3 * n, kThreads), kThreads, 0, st>>>(rdst, 3 * n, d.err);
  k_check_finite<<<grid_for(3 * n, kThreads), kThreads, 0, st>>>(vdst, 3 * n, d.err);
  k_iota<<<grid_for(n, kThreads), kThreads, 0, st>>>(d.id, n);
  OTF_LAUNCH_CHECK();
  if (!h->fp64) {
    k_init_df<<<grid_for(n, kThreads), kThreads, 0, st>>>(d);
    OTF_LAUNCH_CHECK();
  }
  // correlators (their allocations overlap the input copies when the caller's
  // host arrays are pinned): stress and heat flux have 3 series per replica, the
  // velocity correlator 3n series in 3 groups (single system)
  // and the mass-flux cross correlator 6 series per replica
  const corr_spec *specs[kNBanks] = {&p->stress, &p->heatflux, &p->vacf, &p->massflux};
  for (int k = 0; k < kNBanks; ++k) {
    if (specs[k]->u <= 0) continue;
    const int64_t ns = k == 2 ? 3 * n : (k == 3 ? 6 : 3) * (int64_t)count;
    corr_params cp{specs[k]->b, specs[k]->p, specs[k]->m, k == 3 ? 1 : 0, ns, k == 2 ? n : 1,
                   k == 2 ? p->precision : MD_PREC_FP64, specs[k]->u * p->dt};
    Correlator &c = h->banks[k].c;
    h->bank_on[k] = true;
    // the velocity correlator's ring (3.1 GB at 2,048,000 atoms) is zeroed
    // on the side stream, beside the first sort, list build and forces
    int rc = c.create(cp, st, k == 2 ? h->side : nullptr);
    if (rc) return rc;
    if (k == 2) OTF_CUDA(cudaEventRecord(h->ev_ring, h->side));
    c.borrowed = true;
    c.host_steps = &h->steps_done;
    if (k == 2) {
      c.before_read = flush_vacf;
      c.read_ctx = h;
    }
    c.host_base = &h->corr_base;
    c.u = specs[k]->u;
  }
  // the copies from the caller's arrays are done and their values finite
  // before anything works on them (check_device synchronises the stream)
  if (int rc0 = check_device(h)) return rc0;
  // initial layout, forces and observables
  int rc = h->fp64 ? launch_rebuild<double>(h, st) : launch_rebuild<float>(h, st);
  if (rc) return rc;
  if (p->potential == MD_POT_BUCK_EWALD) {
    SpmeParams sp;
    sp.K = p->mesh;
    sp.order = p->order;
    sp.L = h->reps[0].L;
    sp.alpha = p->ewald_alpha;
    sp.ke = p->coulomb;
    if ((rc = h->spme.create(sp, h->fp64, st))) return rc;
  }
  rc = h->fp64 ? launch_pair<double>(h, st) : launch_pair<float>(h, st);
  if (rc) return rc;
  if (h->bank_on[2]) OTF_CUDA(cudaStreamWaitEvent(st, h->ev_ring, 0));  // before any push or readout
  if ((rc = refresh_obs(h))) return rc;
  if ((rc = check_device(h))) return rc;
  if (p->autotune) {
    rc = h->fp64 ? autotune<double>(h) : autotune<float>(h);
    if (rc) return rc;
    if ((rc = refresh_obs(h))) return rc;
    if ((rc = check_device(h))) return rc;
  }
  return MD_OK;
}

void fill_obs(const md_handle *h, int r, md_obs *out) {
  const ObsDev &o = h->h_obs[r];
  out->step = h->h_st->step;
  out->U = o.U;
  out->K = o.K;
  out->T = o.T;
  for (int a = 0; a < 6; ++a) out->sigma[a] = o.sigma[a];
  for (int a = 0; a < 3; ++a) out->q[a] = o.q[a];
  out->T_mean = o.Tn > 0 ? o.Tsum / (double)o.Tn : o.T;
  out->rebuilds = h->h_st->rebuilds;
  for (int a = 0; a < 3; ++a) out->j[a] = o.j[a];
}

int fetch_obs(md_handle *h) {
  OTF_CUDA(cudaMemcpyAsync(h->h_obs, h->d.obs, h->nrep * sizeof(ObsDev), cudaMemcpyDeviceToHost, h->stream));
  OTF_CUDA(cudaMemcpyAsync(h->h_st, h->d.st, sizeof(StepDev), cudaMemcpyDeviceToHost, h->stream));
  OTF_CUDA(cudaStreamSynchronize(h->stream));
  return MD_OK;
}

int scale_impl(md_handle *h) {
  OTF_CUDA(cudaMemcpyAsync(h->d_lam, h->h_lam, h->nrep * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  if (h->fp64)
    k_scale_v<double><<<grid_for(3 * h->d.n, kThreads), kThreads, 0, h->stream>>>(h->d);
  else
    k_scale_v<float><<<grid_for(3 * h->d.n, kThreads), kThreads, 0, h->stream>>>(h->d);
  OTF_LAUNCH_CHECK();
  int rc = refresh_obs(h);
  if (rc) return rc;
  OTF_CUDA(cudaStreamSynchronize(h->stream));
  return MD_OK;
}

int create_handle(const md_params *p, const md_replica *reps, int count, int mem, void *cuda_stream,
                  md_handle **out) {
  *out = nullptr;
  int rc = validate_params(p);
  if (!rc) rc = validate_replicas(p, reps, count, mem);
  if (rc) return rc;
  md_handle *h = new (std::nothrow) md_handle;
  if (!h) return MD_ENOMEM;
  h->stream = (cudaStream_t)cuda_stream;
  rc = init_impl(h, p, reps, count, mem);
  if (rc) {
    release(h);
    return rc;
  }
  *out = h;
  return MD_OK;
}

}  // namespace

extern "C" {

int md_init(const md_params *p, const md_system *s, void *cuda_stream, md_handle **out) {
  clear_error();
  if (!out || !p || !s) {
    set_error("md_init: null argument");
    return MD_EINVAL;
  }
  *out = nullptr;
  if (p->n < 2 || p->n >= (1 << 26) || !(p->box > 0)) {
    set_error("md_init: n must be in [2, 2^26) and box positive");
    return MD_EINVAL;
  }
  if (!s->r || !s->v) {
    set_error("md_init: system needs r, v and a valid mem flag");
    return MD_EINVAL;
  }
  const md_replica one{p->n, p->box, s->r, s->v, s->type};
  return create_handle(p, &one, 1, s->mem, cuda_stream, out);
}

int md_init_replicas(const md_params *p, const md_replica *reps, int32_t count, int32_t mem, void *cuda_stream,
                     md_handle **out) {
  clear_error();
  if (!out) {
    set_error("md_init_replicas: null output handle");
    return MD_EINVAL;
  }
  return create_handle(p, reps, count, mem, cuda_stream, out);
}

int md_step(md_handle *h, int64_t nsteps) {
  clear_error();
  if (!h || nsteps < 0) {
    set_error("md_step: null handle or negative nsteps");
    return MD_EINVAL;
  }
  if (nsteps == 0) return MD_OK;
  int rc = MD_OK;
  if (!h->prm.use_graph) {
    for (int64_t s = 0; s < nsteps && !rc; ++s) rc = step_once(h, h->stream, true);
    if (!rc) rc = join_vacf(h, h->stream);
  } else if (h->timing) {
    // the production graphs with event records inside; set k is read (which
    // waits for its previous replay) while set k ^ 1 is queued behind it;
    // the remainder of the call is one timed graph of that many steps
    int64_t s = 0;
    cudaGraphExec_t gx = nullptr;
    for (int k = 0; s + kGraphSteps <= nsteps && !rc; s += kGraphSteps, k ^= 1) {
      if ((rc = read_timed(h, k)) || (rc = timed_graph_of(h, k, &gx)) || (rc = launch_graph(gx, h->stream))) break;
      h->tev_pending[k] = true;
    }
    const int rem = (int)(nsteps - s);
    if (!rc && rem > 0 && !(rc = read_timed(h, 1 + rem)) && !(rc = timed_graph_of(h, 1 + rem, &gx)) &&
        !(rc = launch_graph(gx, h->stream)))
      h->tev_pending[1 + rem] = true;
    for (int k = 0; k < md_handle::kTimedSets && !rc; ++k) rc = read_timed(h, k);
  } else {
    // whole kGraphSteps-step graphs, then one graph for the remainder
    int64_t s = 0;
    cudaGraphExec_t gx = nullptr;
    for (; s + kGraphSteps <= nsteps && !rc; s += kGraphSteps)
      if (!(rc = graph_of(h, kGraphSteps, &gx))) rc = launch_graph(gx, h->stream);
    const int rem = (int)(nsteps - s);
    if (!rc && rem > 0 && !(rc = graph_of(h, rem, &gx))) rc = launch_graph(gx, h->stream);
  }
  if (rc) return rc;
  // velocity pushes short of a full block stay in their input slots; they
  // are applied by the next call's passes or before the next readout
  // (flush_vacf)
  h->steps_done += nsteps;
  rc = check_device(h);
  if (h->timing && !rc) {
    // pair up the events of each class: (start, stop)
    for (size_t e = 0; e + 1 < h->ev_used; e += 2) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, h->ev[e], h->ev[e + 1]) == cudaSuccess) {
        h->kms[h->ev_class[e]] += ms;
        h->klaunch[h->ev_class[e]] += 1;
      }
    }
  }
  h->ev_used = 0;
  return rc;
}

int md_observables(md_handle *h, md_obs *out) { return md_replica_observables(h, 0, out); }

int md_replica_observables(md_handle *h, int32_t r, md_obs *out) {
  clear_error();
  if (!h || !out || r < 0 || r >= h->nrep) {
    set_error("md_replica_observables: bad argument");
    return MD_EINVAL;
  }
  int rc = fetch_obs(h);
  if (rc) return rc;
  fill_obs(h, r, out);
  return MD_OK;
}

int md_replica_observables_all(md_handle *h, md_obs *out, int32_t count) {
  clear_error();
  if (!h || !out || count != h->nrep) {
    set_error("md_replica_observables_all: null argument or count != %d replicas", h ? h->nrep : 0);
    return MD_EINVAL;
  }
  int rc = fetch_obs(h);
  if (rc) return rc;
  for (int r = 0; r < count; ++r) fill_obs(h, r, out + r);
  return MD_OK;
}

int md_get_particles(md_handle *h, double *r, double *v, double *F, double *epot, double *W, int32_t mem) {
  clear_error();
  if (!h || (mem != MD_MEM_HOST && mem != MD_MEM_DEVICE)) {
    set_error("md_get_particles: bad argument");
    return MD_EINVAL;
  }
  const int64_t n = h->d.n;
  cudaStream_t st = h->stream;
  if (mem == MD_MEM_DEVICE) {
    if (h->fp64)
      k_unsort<double><<<grid_for(n, kThreads), kThreads, 0, st>>>(h->d, r, v, F, epot, W);
    else
      k_unsort<float><<<grid_for(n, kThreads), kThreads, 0, st>>>(h->d, r, v, F, epot, W);
    OTF_LAUNCH_CHECK();
    OTF_CUDA(cudaStreamSynchronize(st));
    return MD_OK;
  }
  if (!h->d_out) OTF_CUDA(cudaMalloc(&h->d_out, 16 * n * sizeof(double)));
  double *o = h->d_out;
  double *dr = o, *dv = o + 3 * n, *dF = o + 6 * n, *de = o + 9 * n, *dW = o + 10 * n;
  if (h->fp64)
    k_unsort<double><<<grid_for(n, kThreads), kThreads, 0, st>>>(h->d, dr, dv, dF, de, dW);
  else
    k_unsort<float><<<grid_for(n, kThreads), kThreads, 0, st>>>(h->d, dr, dv, dF, de, dW);
  OTF_LAUNCH_CHECK();
  const size_t b3 = 3 * n * sizeof(double);
  if (r) OTF_CUDA(cudaMemcpyAsync(r, dr, b3, cudaMemcpyDeviceToHost, st));
  if (v) OTF_CUDA(cudaMemcpyAsync(v, dv, b3, cudaMemcpyDeviceToHost, st));
  if (F) OTF_CUDA(cudaMemcpyAsync(F, dF, b3, cudaMemcpyDeviceToHost, st));
  if (epot) OTF_CUDA(cudaMemcpyAsync(epot, de, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (W) OTF_CUDA(cudaMemcpyAsync(W, dW, 2 * b3, cudaMemcpyDeviceToHost, st));
  OTF_CUDA(cudaStreamSynchronize(st));
  return MD_OK;
}

int md_scale_velocities(md_handle *h, double lambda) {
  clear_error();
  if (!h || !std::isfinite(lambda)) {
    set_error("md_scale_velocities: bad argument");
    return MD_EINVAL;
  }
  for (int k = 0; k < h->nrep; ++k) h->h_lam[k] = lambda;
  return scale_impl(h);
}

int md_replica_scale_velocities(md_handle *h, const double *lambda) {
  clear_error();
  if (!h || !lambda) {
    set_error("md_replica_scale_velocities: null argument");
    return MD_EINVAL;
  }
  for (int k = 0; k < h->nrep; ++k) {
    if (!std::isfinite(lambda[k])) {
      set_error("md_replica_scale_velocities: non-finite factor for replica %d", k);
      return MD_EINVAL;
    }
    h->h_lam[k] = lambda[k];
  }
  return scale_impl(h);
}

int md_reset_correlators(md_handle *h) {
  clear_error();
  if (!h) return MD_EINVAL;
  for (int k = 0; k < kNBanks; ++k)
    if (h->bank_on[k]) {
      int rc = h->banks[k].c.reset();
      if (rc) return rc;
    }
  // correlator base := current step; temperature means restart
  int rc = fetch_obs(h);
  if (rc) return rc;
  h->h_st->corr_base = h->h_st->step;
  h->h_st->vacf_done = 0;
  h->h_st->vacf_ctas = 0u;
  for (int k = 0; k < h->nrep; ++k) {
    h->h_obs[k].Tsum = 0.0;
    h->h_obs[k].Tn = 0;
  }
  OTF_CUDA(cudaMemcpyAsync(h->d.st, h->h_st, sizeof(StepDev), cudaMemcpyHostToDevice, h->stream));
  OTF_CUDA(cudaMemcpyAsync(h->d.obs, h->h_obs, h->nrep * sizeof(ObsDev), cudaMemcpyHostToDevice, h->stream));
  OTF_CUDA(cudaStreamSynchronize(h->stream));
  h->corr_base = h->steps_done;
  return MD_OK;
}

int md_corr(md_handle *h, int32_t which, corr_handle **out) {
  clear_error();
  if (!h || !out || which < 0 || which >= kNBanks) {
    set_error("md_corr: bad argument");
    return MD_EINVAL;
  }
  if (!h->bank_on[which]) {
    set_error("md_corr: correlator %d is disabled (u = 0)", which);
    return MD_EINVAL;
  }
  *out = &h->banks[which];
  return MD_OK;
}

int md_get_config(md_handle *h, md_config *out) {
  clear_error();
  if (!h || !out) {
    set_error("md_get_config: null argument");
    return MD_EINVAL;
  }
  out->replicas = h->nrep;
  out->atoms = h->d.n;
  out->cells = h->d.ncell;
  out->max_neighbors = h->d.maxnb;
  out->pair_threads = h->pair_threads;
  out->build_warps = h->build_warps;
  out->build_kind = h->build_kind;
  out->vacf_input_bytes = (int64_t)h->d.vacf_slots * 3 * h->d.n * (h->fp64 ? sizeof(double) : sizeof(float));
  const bool tiles = h->prm.pair_mode == MD_PAIR_TILES;
  out->tiles = tiles ? h->d.ntiles : 0;
  out->window_capacity = tiles ? h->d.wcap : 0;
  out->tile_threads = tiles ? h->tile_threads : 0;
  for (int a = 0; a < 3; ++a) out->tile_extent[a] = tiles ? h->tile_plans[h->tile_plan].ext[a] : 0;
  if (tiles) out->build_kind = 3;
  return MD_OK;
}

int md_set_timing(md_handle *h, int32_t on) {
  clear_error();
  if (!h) return MD_EINVAL;
  h->timing = on != 0;
  for (int k = 0; k < MD_NKCLASS; ++k) {
    h->kms[k] = 0.0;
    h->klaunch[k] = 0;
  }
  h->ev_used = 0;
  if (h->timing && h->prm.use_graph) {  // the timed graphs, captured before any timed call
    cudaGraphExec_t g = nullptr;
    for (int k = 0; k < md_handle::kTimedSets; ++k) {
      const int rc = timed_graph_of(h, k, &g);
      if (rc) return rc;
    }
  }
  return MD_OK;
}

int md_kernel_times(md_handle *h, double *ms, int64_t *launches) {
  if (!h) return MD_EINVAL;
  for (int k = 0; k < MD_NKCLASS; ++k) {
    if (ms) ms[k] = h->kms[k];
    if (launches) launches[k] = h->klaunch[k];
  }
  return MD_OK;
}

void md_free(md_handle *h) { release(h); }

}  // extern "C"
