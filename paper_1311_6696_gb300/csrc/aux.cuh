// Auxiliary kernels: lattice repacking, norms, var initialisation, observables, CU_0.
#pragma once
#include <utility>
#include "ein.cuh"

namespace peps {

// Per-site gather descriptor for building an oriented lattice from the dense input.
struct OrientSite {
  long long dst;        // element offset of the site tensor in the destination
  int y, x;             // source site
  int du, dl, dn, dr;   // effective dims of the destination legs
  int perm[4];          // destination leg k reads source leg perm[k] (0 u, 1 l, 2 n, 3 r)
};

void orient_lattice(Ctx& cx, const void* src, int src_f32, int Ly, int Lx, int d, int D,
                    const OrientSite* host_sites, int nsites, double* dst);

// (nonzero entries on outward legs, non-finite entries) of a device lattice.
std::pair<long long, long long> input_violations_device(Ctx& cx, const void* src, int src_f32, int Ly, int Lx,
                                                        int d, int D);
// Dominant separable boundaries of the infinite lattice of copies of one tensor
// (given in the four sweep orientations, all legs D), into sigma[4][D][D];
// FLAG_CU0_NOCONV if a side needs more than max_iter steps.
void cu0_infinite(Ctx& cx, const double* const A[4], int d, int D, double* sigma, int max_iter);
// Writes a NaN into element 0 (PEPS_FAULT=nan).
void plant_nan_value(Ctx& cx, void* p, int f32);
// A bounded wait on a flag nothing sets: records FLAG_TIMEOUT in cx.flag after budget_ns.
void wait_unset_flag(Ctx& cx, long long budget_ns);

// All of these act on every problem of their pointer sets (one launch).
// out[0] = ||x||_F (device scalar).
void fro_norm(Ctx& cx, const TP& x, long long n, const TP& out);
// x /= *nrm; if lnacc: *lnacc += log(*nrm).  Sets FLAG_BAD_VALUE on 0 / inf / nan.
void rescale(Ctx& cx, const TP& x, long long n, const TP& nrm, const TP& lnacc);
// Both in sequence; tmp: one device scalar per problem (absent: cx.tmp, one problem).
void normalize(Ctx& cx, const TP& x, long long n, const TP& lnacc, const TP& tmp = TP());

// var start: dst[c,n,o,e] = src[c,n,o,e] where inside src's extent, else
// noise * 1e-3 * ||src|| / sqrt(numel(dst)); noise from SplitMix64 keyed by
// (seed, tag, y, x, flat index of dst).  tmp as for normalize.
void var_init(Ctx& cx, const TP& src, const int sdims[4], const TP& dst, const int ddims[4],
              unsigned long long seed, int tag, int y, int x, const TP& tmp = TP());

// out[i] = sum_ab rho_i[a][b] op[b][a] / sum_a rho_i[a][a] for count matrices k x k.
void expect_batch(Ctx& cx, const double* rho, int count, int k, const double* op, double* out);

// ln_norm = sum(lns[0..nl)) + extra + log|s|, sign = sign(s) (device scalars).
void finish_norm(Ctx& cx, const double* lns, int nl, const double* extra, const double* s,
                 double* out_ln, double* out_sign);

void fill(Ctx& cx, const TP& x, long long n, double v);
void copy(Ctx& cx, const TP& dst, const TP& src, long long n);

// CU_0 separable boundaries of one oriented lattice (Section 5.1), computed
// by one CTA.  Site tensors at `sites` (per-site offsets/dims in `meta`),
// closures as device matrices.  Output: out[r][x] = D x D matrix (stride
// out_stride per row, mat_stride per site) on the up legs of row r, r = 1..Ly-1.
struct Cu0Lattice {
  int Ly, Lx, d, Dmax;
  const double* A;              // site tensors base
  const long long* off;         // [Ly*Lx] element offsets of site tensors
  const int* dims;              // [Ly*Lx*4] du, dl, dn, dr
  const double* top;            // [Lx] closures on row 0 up legs, stride Dmax^2
  const double* left;           // [Ly] closures, stride Dmax^2
  const double* right;          // [Ly]
  double* out;                  // [Ly][Lx][Dmax^2]
  double* work;                 // scratch, see cu0_work_size
  int max_half;
  double tol;
};
size_t cu0_work_size(int Lx, int d, int Dmax);
void cu0_launch(Ctx& cx, const Cu0Lattice* lats, int nlat);

}  // namespace peps
