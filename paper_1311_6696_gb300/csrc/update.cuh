// Tensor update of the full / cluster update (Section 2): alternating least
// squares on the reduced tensors of a bond, N_l A_l = b_l, in FP64.
#pragma once
#include <vector>

#include "ein.cuh"

namespace peps {

// dst = src with its five axes reordered: dst axis k is src axis perm[k]
// (src row-major with extents dims[0..4]).
void permute5(Ctx& cx, const double* src, const int dims[5], const int perm[5], double* dst);

// One bond of a shape group (every bond of a group has the same kl, kr, Do, Dn).
struct BondAls {
  const double* N = nullptr;    // [kl][kr][kl][kr], the norm matrix (ket legs, bra legs)
  const double* al = nullptr;   // [kl][d][Do], reduced left tensor before the gate
  const double* ar = nullptr;   // [kr][d][Do], reduced right tensor before the gate
  double* al_new = nullptr;     // out: [kl][d][Dn]
  double* ar_new = nullptr;     // out: [Dn][d][kr]
  double* q = nullptr;          // out: q[0] = <psi-Theta|N|psi-Theta>, q[1] = <Theta|N|Theta>
};

// Gate (device, (d*d) x (d*d) row-major, G[(s t),(s' t')]) applied to every
// bond of the group, then `iters` ALS rounds (left solve, right solve) with
// the positive part of the symmetrised N, then the balanced split.  The
// Cholesky systems have kl*Dn and kr*Dn unknowns per physical value; both must
// be <= kCholMax.
constexpr int kCholMax = 160;
void bond_als(Ctx& cx, int d, int kl, int kr, int Do, int Dn, const double* gate, const std::vector<BondAls>& bonds,
              int iters);

// Writes an updated oriented site tensor (extents s, u, l, n, r of the
// orientation) into site (y, x) of a dense lattice [Ly][Lx][d][D][D][D][D]
// (FP64 or FP32), zero beyond the tensor's extents; oriented leg k is dense
// leg perm[k] (0 u, 1 l, 2 n, 3 r).
struct SiteStore {
  const double* src;
  int y, x;
  int dims[5];
  int perm[4];
};
void store_sites(Ctx& cx, void* dst, int dst_f32, int Lx, int d, int D, const std::vector<SiteStore>& sites);

}  // namespace peps
