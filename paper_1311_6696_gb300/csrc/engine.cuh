// Host-side orchestration of the boundary-MPS contraction (device resident).
// An engine runs nb independent problems of identical shape in lockstep (the
// cluster windows of one shape; nb = 1 for the full lattice): every tensor is
// a pointer set (TP) with one pointer per problem, and every step is one
// batched launch for all of them.
#pragma once
#include <functional>
#include <memory>
#include <vector>

#include "ein.cuh"

namespace peps {

struct SiteT {
  TP p;
  int d = 0, du = 0, dl = 0, dn = 0, dr = 0;
  Dims dims() const { return {d, du, dl, dn, dr}; }
};

struct Mat {
  TP p;                        // n x n, row-major (ket leg, bra leg)
  int n = 0;
};

// A (sub-)lattice in one orientation, with a closure matrix on every outward leg.
struct OLat {
  int Ly = 0, Lx = 0, d = 0;
  std::vector<SiteT> sites;    // row-major
  std::vector<Mat> top, bottom, left, right;
  const SiteT& at(int y, int x) const { return sites[size_t(y) * Lx + x]; }
};

struct Mps {
  std::vector<TP> p;
  std::vector<Dims> dims;      // [a, u, v, b]
  bool right_canonical = false;   // sites 1..L-1 right-orthonormal, centre at site 0
};

struct Opts {
  int chi = 16;
  int mode = PEPS_SVD;
  int sweeps = 2;
  int precision = PEPS_PREC_FP64;
  unsigned long long seed = 0;
};

// Everything a full or cluster environment keeps on the device.
struct EnvData {
  int Ly = 0, Lx = 0, d = 0, D = 0;
  bool has_norm = false;
  double* rho_site = nullptr;   // [Ly*Lx][d*d]
  double* rho_h = nullptr;      // [Ly*(Lx-1)][d^4]
  double* rho_v = nullptr;      // [(Ly-1)*Lx][d^4]
  double* lnnorm = nullptr;     // [2]: ln|N|, sign
};

// Contraction engine bound to one stream/workspace.
class Engine {
 public:
  Engine(Ctx& cx, const Opts& o, int d, int Dmax, int Lmax, int nb = 1);
  ~Engine();
  // A second stream (and its own chain buffers) on which row_rhos builds the
  // right environments while the left ones are built on the main stream.
  // Taken only when one more buffer set is small (single problem, < 512 MB).
  void enable_dual(cudaStream_t st2);

  // Top-down boundaries of `lat`: out[y] = boundary above row y, y = 0..upto.
  // lnacc (a device scalar per problem) accumulates the log of every rescaling factor.
  // on_boundary(y, out[y]), if given, is called as soon as out[y] is enqueued.
  std::vector<Mps> sweep(const OLat& lat, int tag, int upto, const TP& lnacc, Arena& keep,
                         const std::function<void(int, const Mps&)>& on_boundary = nullptr);

  // Density matrices of row y between top boundary T and bottom boundary B:
  // rho_site of column x into dst for every (x, dst) in `sites`, rho of the
  // bond (x, x+1) into dst for every (x, dst) in `bonds`.
  using Targets = std::vector<std::pair<int, TP>>;
  void row_rhos(const OLat& lat, const Mps& T, const Mps& B, int y, const Targets& sites,
                const Targets& bonds);

  // The tensor update of the full update (Section 2, reduced tensors): for the
  // pair (x, x+1) of row y, each site is split by a QR into an isometry and a
  // reduced tensor, A(x) = X_l a_l over the legs (u l n) | (s r) and
  // A(x+1) = X_r a_r over (u n r) | (t l), and the norm network with a_l, a_r
  // and their conjugates removed is contracted into N[kl][kr][kl][kr]: the
  // bond density-matrix network with the isometries in place of the sites.
  struct BondNorm {
    int x = 0;                          // left column of the pair
    double* ml = nullptr;               // scratch: the left site as (u l n) x (s r)
    double* mr = nullptr;               // scratch: the right site as (u n r) x (t l)
    double* xl = nullptr;               // [kl][u l n]
    double* xr = nullptr;               // [kr][u n r]
    double* al = nullptr;               // [kl][s][r]
    double* ar = nullptr;               // [kr][t][l]
    double* N = nullptr;                // [kl][kr][kl][kr]
  };
  void row_bond_norms(const OLat& lat, const Mps& T, const Mps& B, int y, const std::vector<BondNorm>& bonds);

  // ln|<psi|psi>| from the top boundary above the last row (writes out[0], out[1] = sign).
  void norm_from_top(const OLat& lat, const Mps& T, const TP& lns_acc, const TP& out);

  int problems() const { return nb_; }
  // Run the next calls on the first B problems only (B <= the engine's capacity).
  void use(int B);
  // Device doubles one problem of an engine with these settings holds.
  static size_t footprint(const Opts& o, int d, int Dmax, int Lmax);

  Ctx& cx;
  Opts opt;

 private:
  Mps closure_mps(const std::vector<Mat>& mats, Arena& keep);
  // Row environments of row y: Lenv_[x] for x < xmax, Renv_[x] for x >= xmin.
  void row_envs(const OLat& lat, const Mps& T, const Mps& B, int y, int xmin, int xmax, std::vector<Dims>& ld,
                std::vector<Dims>& rd);
  // Site tensor A at column x with its physical pair open: W[e,r,q,b,s,t]
  // (pushed in from the left, into bb_) and V[a,l,m,k,s,t] (from the right, into vv_).
  Dims open_left(const Mps& T, const Mps& B, int x, const SiteT& A, const Dims& ldx);
  Dims open_right(const Mps& T, const Mps& B, int x, const SiteT& A, const Dims& rdx);
  Mps absorb_compress(const Mps& T, const OLat& lat, int y, int tag, const TP& lnacc, Arena& keep);
  Mps product_mps(const Mps& T, const OLat& lat, int y, Arena& keep);
  void left_canonicalize(Mps& P, Arena& keep);
  void svd_truncate(Mps& P, const std::vector<int>& caps, Arena& keep);
  Mps var_compress(const Mps& T, const OLat& lat, int y, const std::vector<int>& caps, int tag,
                   int& centre, Arena& keep);

  // One pairwise contraction.  FP64 mode: FP64 gather-GEMM, every operand FP64.
  // Tensor-core modes: tcgen05 GEMM; a64/b64/c64 tag each tensor FP64 (else FP32).
  // b_site: B is a site tensor (unchanged during the call): its packed copy is cached.
  void con(const char* spec, const TP& A, bool a64, const Dims& ad, const TP& B, bool b64, const Dims& bd,
           const TP& C, bool c64, bool b_site = false);
  std::unique_ptr<PackCache> site_packs_;
  // `per` doubles for every problem from arena a.
  TP alloc(Arena& a, size_t per) const;
  bool tc_ = false;   // tensor-core contractions (chain intermediates stored FP32)
  bool x64_ = true;   // dtype of the chain intermediates X1, X2, X3

  // absorb chain pieces
  Dims chain_left(const TP& L, const Dims& ld, const TP& M, const Dims& md, const SiteT& A, const TP& X3);
  Dims chain_right(const TP& R, const Dims& rd, const TP& M, const Dims& md, const SiteT& A, const TP& Y3);

  // The stream, scratch, chain buffers and pack cache the contraction helpers use.
  struct Side {
    Ctx* cx;
    TP X1, X2, X3, tmp;
    PackCache* cache;
    size_t x1n, x2n;   // doubles from X1.p[0] / X2.p[0] (contiguous over the problems)
  };
  // Tensor-core absorb chains: each GEMM writes the next one's operand.
  // open: the bra stage keeps the physical index open (X3 / Y3 of a site's density matrix).
  Dims chain_left_tc(const TP& L, const Dims& ld, const TP& M, const Dims& md, const SiteT& A, const TP& X3,
                     bool open);
  Dims chain_right_tc(const TP& R, const Dims& rd, const TP& M, const Dims& md, const SiteT& A, const TP& Y3,
                      bool open);
  Side main_, aux_;
  Side* side_ = &main_;
  bool dual_ = false;
  std::unique_ptr<Arena> ws2_;
  std::unique_ptr<Ctx> cx2_;
  std::unique_ptr<PackCache> cache2_;
  cudaStream_t ws2_stream_ = nullptr;

  int d_, Dmax_, Lmax_, nb_, cap_;
  size_t x1per_ = 0, x2per_ = 0;   // doubles per problem of X1_ / X2_ (their stride)
  size_t bigN_;                 // chi^2 * Dmax^4 (elements of the largest chain intermediate / d)
  TP X1_, X2_, X3_, bb_, vv_;   // chain buffers; bb_, vv_: local vector / open-site tensors
  std::vector<TP> Lenv_, Renv_;
  size_t envN_;
  TP one_;                      // device scalar 1.0 (shared)
  TP tmp0_, tmp1_;              // one device scalar per problem each
};

// Caps of the new boundary (same rule as the documented reading).
std::vector<int> bond_caps(const std::vector<int>& phys, const std::vector<long long>& prod, int chi);

}  // namespace peps
