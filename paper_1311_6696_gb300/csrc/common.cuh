// Internal helpers shared by the library's translation units: error type,
// stream-ordered arenas, kernel-class instrumentation.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/peps.h"

namespace peps {

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define PEPS_CUDA(x)                                                                   \
  do {                                                                                 \
    cudaError_t e_ = (x);                                                              \
    if (e_ != cudaSuccess)                                                             \
      throw ::peps::Error(e_ == cudaErrorMemoryAllocation ? PEPS_ENOMEM : PEPS_ECUDA,   \
                          std::string(#x) + ": " + cudaGetErrorString(e_));            \
  } while (0)

#define PEPS_CHECK_LAUNCH() PEPS_CUDA(cudaGetLastError())

#define PEPS_REQUIRE(cond, msg)                                                        \
  do {                                                                                 \
    if (!(cond)) throw ::peps::Error(PEPS_EINVAL, msg);                                \
  } while (0)

// ---------------------------------------------------------------------------
// Kernel classes for instrumentation.
// ---------------------------------------------------------------------------
enum KClass {
  K_GEMM_F64 = 0,   // gather-GEMM, FP64 (absorb chain, envs, density matrices)
  K_GEMM_TC,        // tcgen05 GEMM (TF32 / BF16 absorb chain)
  K_QR,             // Householder / Cholesky QR (FP64)
  K_SVD,            // one-sided Jacobi SVD (FP64)
  K_CU0,            // CU_0 separable boundary fixed point
  K_OBS,            // local observables
  K_AUX,            // init noise, norms, rescale, copies, reductions
  K_PACK,           // operand repacking for the tensor cores (gather + TF32/BF16 split)
  K_NCLASS
};

void prof_launch(KClass c, cudaStream_t st, double flops, double bytes);
void prof_done(KClass c, cudaStream_t st);
void prof_more(KClass c, int kernels);
bool prof_timing();

// RAII helper: record around one launch.
struct Launch {
  KClass c;
  cudaStream_t st;
  Launch(KClass c_, cudaStream_t st_, double flops = 0, double bytes = 0) : c(c_), st(st_) {
    prof_launch(c, st, flops, bytes);
  }
  ~Launch() { prof_done(c, st); }
  // The scope counts as one kernel launch; a scope that launches more kernels
  // adds them here, so the counters hold kernel launches, not scopes.
  void more(int kernels = 1) { prof_more(c, kernels); }
};

// ---------------------------------------------------------------------------
// Iteration caps and host-side fault injection.
//   Caps (peps_set_iteration_caps): half-sweeps of a CU_0 fixed point and
//   sweeps of a one-sided Jacobi SVD; a computation that hits one fails with
//   PEPS_ECONVERGE.  Process-wide; a recorded plan keeps the caps it was
//   recorded with.
//   Faults (environment variable PEPS_FAULT, read at the start of every call;
//   for tests of the error paths, nothing here touches the GPU's state):
//     alloc     every device allocation of the call fails   -> PEPS_ENOMEM
//     nan       a NaN is planted in the call's device copy of the lattice
//               before validation                           -> PEPS_EINVAL
//     converge  both caps are 1 for the call                -> PEPS_ECONVERGE
//               (wherever an iteration does not stop in one step)
// ---------------------------------------------------------------------------
enum Fault { FAULT_NONE = 0, FAULT_ALLOC = 1, FAULT_NAN = 2, FAULT_CONVERGE = 3 };
int fault_from_env();
int cap_cu0_half_sweeps();
int cap_jacobi_sweeps();
extern std::atomic<int> g_fault_alloc;      // > 0 while a PEPS_FAULT=alloc call runs

// ---------------------------------------------------------------------------
// Stream-ordered bump arena (cudaMallocAsync chunks, freed together).
// ---------------------------------------------------------------------------
class Arena {
 public:
  // async: chunks come from cudaMallocAsync on `st` and are freed stream-ordered;
  // otherwise cudaMalloc / cudaFree (for memory that outlives the caller's stream).
  explicit Arena(cudaStream_t st, size_t chunk = size_t(64) << 20, bool async = true)
      : st_(st), chunk_(chunk), async_(async) {}
  ~Arena() { release(); }
  Arena(const Arena&) = delete;
  Arena& operator=(const Arena&) = delete;

  void* alloc(size_t bytes) {
    std::lock_guard<std::mutex> g(mu_);   // shared by lane threads when it owns an env
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    if (g_fault_alloc.load(std::memory_order_relaxed) > 0)
      throw Error(PEPS_ENOMEM, "device allocation failed (injected: PEPS_FAULT=alloc)");
    if (bytes > left_) {
      size_t n = bytes > chunk_ ? bytes : chunk_;
      void* p = nullptr;
      cudaError_t e = async_ ? cudaMallocAsync(&p, n, st_) : cudaMalloc(&p, n);
      if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(PEPS_ENOMEM, std::string("device allocation of ") + std::to_string(n) +
                                     " bytes failed: " + cudaGetErrorString(e));
      }
      chunks_.push_back(p);
      cur_ = static_cast<char*>(p);
      left_ = n;
      total_ += n;
    }
    void* r = cur_;
    cur_ += bytes;
    left_ -= bytes;
    return r;
  }
  double* dalloc(size_t n) { return static_cast<double*>(alloc(n * sizeof(double))); }
  float* falloc(size_t n) { return static_cast<float*>(alloc(n * sizeof(float))); }
  void release() {
    std::lock_guard<std::mutex> g(mu_);
    for (void* p : chunks_) {
      if (async_)
        cudaFreeAsync(p, st_);
      else
        cudaFree(p);
    }
    chunks_.clear();
    cur_ = nullptr;
    left_ = 0;
  }
  size_t total() const { return total_; }
  cudaStream_t stream() const { return st_; }

 private:
  cudaStream_t st_;
  size_t chunk_;
  bool async_;
  std::vector<void*> chunks_;
  char* cur_ = nullptr;
  size_t left_ = 0;
  size_t total_ = 0;
  std::mutex mu_;
};

// Records `msg` as this thread's last error (peps_last_error) and returns `code`.
int peps_set_error(int code, const std::string& msg);

inline unsigned cdiv(long long a, long long b) { return unsigned((a + b - 1) / b); }

}  // namespace peps
