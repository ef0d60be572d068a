// Smooth particle-mesh Ewald on the GPU: the reciprocal-space energy, forces
// and per-particle virial of point charges in a cubic box (Essmann et al.
// 1995, the method of arXiv 2503.07526 Sec. 5.3), with the per-particle split
// of Appendix B.
#pragma once

#include <cufft.h>

#include "common.cuh"

namespace otf {

struct SpmeParams {
  int K = 0;          // mesh points per side
  int order = 8;      // B-spline order (even, 4..8)
  double L = 0.0;     // box side
  double alpha = 0.0; // Ewald splitting parameter
  double ke = 1.0;    // Coulomb constant
};

// Atoms as the MD engine holds them: cell-sorted, each with a packed cell
// index (x | y << 10 | z << 20), its offset from the cell centre (the Vec4
// record of the pair type, whose w holds the charge; in the mixed form the
// offset's low words are in rlo [n]) and a cell edge.
struct SpmeAtoms {
  int64_t n = 0;
  const int *cpk = nullptr;
  const void *rel = nullptr;
  const float4 *rlo = nullptr;
  double edge = 0.0;
  const int *cellstart = nullptr;  // [nc^3 + 1]: atoms of cell c are [cellstart[c], cellstart[c+1])
  int nc = 0;                      // cells per side
};

class Spme {
 public:
  int create(const SpmeParams &p, bool fp64, cudaStream_t st);
  void destroy();
  // Adds, per atom, the reciprocal-space force, energy and virial and the
  // self energy -ke alpha q^2 / sqrt(pi) to F [3][n], epot [n], W [6][n]
  // (arrays of the pair type: float in the mixed form, double in FP64).
  int run(const SpmeAtoms &a, void *F, void *epot, void *W, cudaStream_t st);
  bool on() const { return Qi_ != nullptr; }

 private:
  template <typename T>
  int run_t(const SpmeAtoms &a, T *F, T *epot, T *W, cudaStream_t st);
  SpmeParams p_;
  bool fp64_ = false;
  unsigned long long *Qi_ = nullptr;  // fixed-point charge mesh (deterministic sums)
  void *Qr_ = nullptr;                // real mesh [K^3]
  void *G1_ = nullptr, *G2_ = nullptr;  // half spectra [K][K][K/2+1]
  void *phi_ = nullptr, *psi_ = nullptr;  // convolved meshes [K^3]
  void *bmod_ = nullptr;              // |b(m)|^2 [K]
  cufftHandle fwd_ = 0, inv_ = 0;
  bool plans_ = false;
  bool attr_ = false;  // shared-memory limits raised for the tile kernels
};

}  // namespace otf
