// Pairwise tensor contractions ("einsum" of two operands) on the GPU.
#pragma once
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
void ein(Ctx& cx, const char* spec, const double* A, const Dims& ad, const double* B,
         const Dims& bd, double* C, double alpha = 1.0, double beta = 0.0);

// C = alpha * contract(A, B) on the tensor cores (tcgen05): operands are
// FP64 (x_f64 = 1) or FP32 tensors, repacked to TF32 / BF16; C is written as
// FP64 or FP32 in any index order; with Clo (FP32 output only) C receives the
// TF32-rounded value and Clo the rounded residual.  prec is PEPS_PREC_*.
void ein_tc(Ctx& cx, const char* spec, const void* A, int a_f64, const Dims& ad, const void* B, int b_f64,
            const Dims& bd, void* C, int c_f64, int prec, double alpha = 1.0, void* Clo = nullptr);
int tc_available();

}  // namespace peps
