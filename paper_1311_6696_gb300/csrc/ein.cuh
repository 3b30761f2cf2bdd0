// Pairwise tensor contractions ("einsum" of two operands) on the GPU.
#pragma once
#include <cstddef>
#include <initializer_list>
#include <map>
#include <string>
#include <vector>

#include "common.cuh"

namespace peps {

// Per-call execution context: stream, persistent workspace and a reusable
// scratch buffer (stream ordered, so consecutive launches may reuse it).
struct Ctx {
  cudaStream_t st;
  Arena* ws;
  double* scr = nullptr;
  size_t scr_n = 0;
  int* flag = nullptr;   // device status word (ECONVERGE / ETIMEOUT), zeroed per call
  double* tmp = nullptr; // 8 device doubles for short-lived scalars (stream ordered)
  // Set while the call is being recorded into a CUDA graph: memory that host
  // data is copied into comes from here (allocated once, kept by the graph's owner).
  Arena* persist = nullptr;
  // Largest thread-block cluster a QR may use (0: no limit beyond 16).
  int qr_cmax = 0;
  // Iteration caps of this call (Jacobi SVD sweeps, CU_0 half-sweeps).
  int svd_cap = 60;
  int cu0_cap = 200;
  // Instrumentation of FP64 contractions that are part of a factorisation:
  // class to charge (-1: their own) and whether to count their flops.
  int f64_class = -1;
  bool f64_flops = true;

  Ctx(cudaStream_t s, Arena* w) : st(s), ws(w) {}
  ~Ctx() {
    if (scr) cudaFreeAsync(scr, st);
  }
  double* scratch(size_t n) {
    if (n > scr_n) {
      if (scr) cudaFreeAsync(scr, st);
      size_t m = n + n / 4 + 1024;
      void* p = nullptr;
      cudaError_t e = cudaMallocAsync(&p, m * sizeof(double), st);
      if (e != cudaSuccess) {
        cudaGetLastError();
        scr = nullptr;
        scr_n = 0;
        throw Error(PEPS_ENOMEM, "scratch allocation failed");
      }
      scr = static_cast<double*>(p);
      scr_n = m;
    }
    return scr;
  }
};

// Independent problems of identical shape that one batched launch serves
// (e.g. the cluster windows of one shape): every tensor argument is a set of
// per-problem device pointers, passed by value in the kernel parameters.
constexpr int MAXB = 64;

struct TP {
  int n = 0;              // 0: absent, 1: one pointer (shared by every problem), else per problem
  void* p[MAXB];
  TP() {}
  TP(std::nullptr_t) {}
  TP(const void* q) : n(q ? 1 : 0) { p[0] = const_cast<void*>(q); }   // one problem
  __host__ __device__ void* v(int b) const { return n == 1 ? p[0] : p[b]; }
  __host__ __device__ double* d(int b) const { return static_cast<double*>(v(b)); }
  bool null() const { return n == 0; }
  // The same element offset (in doubles) into every problem's tensor.
  TP off(long long e) const {
    TP r = *this;
    for (int b = 0; b < n; ++b) r.p[b] = static_cast<double*>(p[b]) + e;
    return r;
  }
  // Every slot filled (a shared pointer repeated), for kernel parameters.
  TP all(int B) const {
    TP r = *this;
    if (n == 1)
      for (int b = 1; b < B; ++b) r.p[b] = p[0];
    r.n = n == 0 ? 0 : B;
    return r;
  }
};

// Per-problem blocks of `per` doubles (rounded up to 32) starting at base.
TP strided(double* base, int count, size_t per);
// Number of problems of a call: every present argument has 1 or B pointers.
int problems(std::initializer_list<const TP*> args);

// Device copy of `bytes` of host data, valid for all later work on cx.st; the
// host buffer may be released when this returns.  While recording a graph the
// copy is made once into cx.persist (it is shape data, fixed for the graph).
void* stage(Ctx& cx, const void* host, size_t bytes);

using Dims = std::vector<int>;

inline size_t numel(const Dims& d) {
  size_t n = 1;
  for (int v : d) n *= size_t(v);
  return n;
}

// Output dims of spec "ab,bc->ac" given operand dims.
Dims ein_dims(const char* spec, const Dims& ad, const Dims& bd);

// C = alpha * sum_{shared} A B + beta * C, all tensors contiguous row-major,
// in FP64.  Indices present in A, B and C are batch indices; indices in only
// one operand must appear in C.
void ein(Ctx& cx, const char* spec, const TP& A, const Dims& ad, const TP& B,
         const Dims& bd, const TP& C, double alpha = 1.0, double beta = 0.0);

// C = alpha * contract(A, B) on the tensor cores (tcgen05): operands are
// FP64 (x_f64 = 1) or FP32 tensors, repacked to TF32 / BF16; C is written as
// FP64 or FP32 in any index order; with Clo (FP32 output only) C receives the
// TF32-rounded value and Clo the rounded residual.  prec is PEPS_PREC_*.
// Packed tensor-core copies of B operands that stay unchanged for the cache's
// lifetime (the site tensors of a call), keyed by contraction, precision and
// the operand's pointers; memory from `mem`.
struct PackCache {
  explicit PackCache(Arena* a) : mem(a) {}
  struct Entry {
    void* hi;
    void* lo;
    long long ld;
  };
  Arena* mem;
  std::map<std::string, Entry> entries;
};

// An operand in the tensor-core layout of one contraction: [np * pad][ld]
// (rows over the contraction's M letters, K contiguous), hi part and, for the
// split precisions, the rounded residual.
struct TcOperand {
  void* hi = nullptr;
  void* lo = nullptr;
  long long ld = 0, pad = 0;
  int np = 0;
};

// Chained contractions without a repack in between.
//   a_pre:    operand A is already in this contraction's layout (written by
//             the previous contraction's epilogue).
//   next:     write C not as a tensor but as operand A of the contraction
//             `next` (whose B operand has dims next_bd), into next_mem
//             (next_cap doubles, contiguous over the problems); next_out
//             receives its description.  C and Clo are then ignored.
// K is ordered as in a plain call, so the result is the same as packing the
// FP32 output of a plain call.
struct TcChain {
  const TcOperand* a_pre = nullptr;
  const char* next = nullptr;
  Dims next_bd;
  double* next_mem = nullptr;
  size_t next_cap = 0;
  TcOperand* next_out = nullptr;
};

// Doubles a TcChain target needs for operand A of `spec` (hi and lo parts).
size_t tc_operand_words(const char* spec, const Dims& ad, const Dims& bd, int np, int prec);

// bcache: B is packed once per cache and reused (B must not change meanwhile).
void ein_tc(Ctx& cx, const char* spec, const TP& A, int a_f64, const Dims& ad, const TP& B, int b_f64,
            const Dims& bd, const TP& C, int c_f64, int prec, double alpha = 1.0, const TP& Clo = TP(),
            PackCache* bcache = nullptr, const TcChain* chain = nullptr);
int tc_available();

}  // namespace peps
