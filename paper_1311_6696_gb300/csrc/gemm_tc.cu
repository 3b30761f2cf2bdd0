// Tensor-core contractions for the absorb chain (TF32 or BF16 inputs, FP32
// accumulation) on sm_103a: tcgen05.mma with the accumulator in TMEM, operand
// tiles staged by TMA (cp.async.bulk.tensor, 128-byte swizzle) through an
// mbarrier ring, one elected thread issuing the MMAs.
//
// C[m, n] = alpha * sum_k A[m, k] B[n, k]: A is [M][K] and B is [N][K], both
// K-contiguous (rows padded to 16 bytes).  The epilogue reads the accumulator
// with tcgen05.ld and writes every element through the same row/column offset
// decomposition as the FP64 gather-GEMM, so the output can be any permutation
// of the (M, N) indices -- the layout the next contraction wants.
//
// Operands that are not already [M][K] / [N][K] are repacked by k_pack (a
// gather copy that also rounds to TF32 / BF16 and, for the split variants,
// writes the residual as a second operand: x ~ hi + lo, product ~ hi*hi +
// hi*lo + lo*hi).
//
// Independent problems of one shape share a launch: problem p's operands are
// packed at rows [p * rows_pad, p * rows_pad + M) of one [P * rows_pad][K]
// array (rows_pad a multiple of the tile height, so no tile straddles two
// problems), and the epilogue writes through problem p's output pointer.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <cstdlib>
#include <string>
#include <vector>

#include "ein.cuh"
#include "linalg.cuh"

namespace peps {
namespace {

constexpr int TC_BM = 128;            // UMMA M (cta_group::1): accumulator row = TMEM lane
constexpr int TC_THREADS = 128;       // 4 warps: TMA producer, MMA issuer, all four read TMEM
constexpr int TC_STAGES = 4;
constexpr int TC_ROWB = 128;          // bytes per tile row = one 128-byte swizzle row
constexpr int MAXG = 8;

struct Grp {
  int n;
  int dim[MAXG];
  long long s[MAXG];
};

struct TcArgs {
  long long M, N, K;
  int ktiles;
  int split;         // 1: A_lo, B_lo present
  int bf16;          // 0: tf32, 1: bf16
  int out_f64;       // 1: C is double, else float
  int out_lo;        // 1: also write C_lo (split residual), C is then the rounded hi part
  int out_tc;        // C is a tensor-core operand of the next contraction: 1 = TF32 (float,
                     // rounded), 2 = BF16; with out_lo the rounded residual goes to C_lo
  int stages;        // ring depth (<= TC_STAGES), chosen to fit shared memory
  int nprob;         // problems in this launch
  int cols_fast;     // 1: the output's unit stride is in the N group (write along columns)
  int splitk;        // > 1: blockIdx.y takes k tiles [y * kt_per, ...) and writes FP32 partials
  int kt_per;
  float* part;       // [splitk][nprob][M][N] partial sums
  long long pad_m, pad_n;   // packed rows per problem (multiples of TC_BM and BN)
  TP C, Clo;         // per problem
  Grp gm, gn;        // output offsets of the M and N groups
  double alpha;
  int* flag;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait (about 2 s of SM clock at 2 GHz); on timeout sets the status
// word and returns false so the caller can drain and leave.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* flag) {
  const long long start = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - start > 4000000000LL) {
      atomicOr(flag, FLAG_TIMEOUT);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(smem_u32(dst)), "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory descriptor of a K-major tile laid out by TMA with 128-byte
// swizzle: 8-row groups 1024 bytes apart (SBO), descriptor version 1, swizzle 2.
__device__ __forceinline__ uint64_t sdesc(const void* tile) {
  const uint64_t a = smem_u32(tile);
  return ((a >> 4) & 0x3FFFull) | (1ull << 16) | (uint64_t(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void decomp(const Grp& g, long long idx, long long& off) {
  off = 0;
  for (int i = g.n - 1; i >= 0; --i) {
    const long long q = idx / g.dim[i];
    off += (idx - q * g.dim[i]) * g.s[i];
    idx = q;
  }
}

// Element o of problem pb's output: FP64, FP32, or a tensor-core operand of
// the next contraction (TF32 or BF16, rounded, with the rounded residual in
// C_lo for the split precisions) -- the values the operand pack would make
// from the FP32 result.
__device__ __forceinline__ void put_out(const TcArgs& g, int pb, long long o, float v) {
  if (g.out_f64) {
    static_cast<double*>(g.C.p[pb])[o] = double(v);
  } else if (g.out_tc == 2) {
    const __nv_bfloat16 h = __float2bfloat16(v);
    static_cast<__nv_bfloat16*>(g.C.p[pb])[o] = h;
    if (g.out_lo) static_cast<__nv_bfloat16*>(g.Clo.p[pb])[o] = __float2bfloat16(v - __bfloat162float(h));
  } else if (g.out_tc == 1 || g.out_lo) {
    const float h = round_tf32(v);
    static_cast<float*>(g.C.p[pb])[o] = h;
    if (g.out_lo) static_cast<float*>(g.Clo.p[pb])[o] = round_tf32(v - h);
  } else {
    static_cast<float*>(g.C.p[pb])[o] = v;
  }
}

// One 128 x BN output tile per CTA.
template <int BN>
__global__ void __launch_bounds__(TC_THREADS) k_gemm_tc(const __grid_constant__ CUtensorMap ta,
                                                        const __grid_constant__ CUtensorMap tb,
                                                        const __grid_constant__ CUtensorMap tal,
                                                        const __grid_constant__ CUtensorMap tbl,
                                                        const TcArgs g) {
  constexpr int A_BYTES = TC_BM * TC_ROWB;
  constexpr int B_BYTES = BN * TC_ROWB;
  extern __shared__ __align__(1024) uint8_t dsm[];
  // 1024-byte aligned stage ring: [A, B, (A_lo, B_lo)] per stage
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~uintptr_t(1023));
  const int stage_bytes = g.split ? 2 * (A_BYTES + B_BYTES) : (A_BYTES + B_BYTES);
  __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES], done;
  __shared__ uint32_t tmem_base;
  __shared__ long long offm[TC_BM], offn[BN];
  __shared__ float stage_out[4][32][17];   // per warp: 32 rows x 16 columns of the accumulator

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long tiles_n = (g.N + BN - 1) / BN;
  const long long tiles = ((g.M + TC_BM - 1) / TC_BM) * tiles_n;
  const int pb = int(blockIdx.x / tiles);
  const long long t = blockIdx.x % tiles;
  const long long m0 = (t / tiles_n) * TC_BM;
  const long long n0 = (t % tiles_n) * BN;
  const int ra = int(pb * g.pad_m + m0), rb = int(pb * g.pad_n + n0);   // packed rows of the tiles

  if (tid == 0) {
    for (int s = 0; s < g.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    const uint32_t ncols = BN < 32 ? 32 : BN;
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  for (int i = tid; i < TC_BM; i += TC_THREADS) {
    const long long m = m0 + i;
    long long o = -1;
    if (m < g.M) decomp(g.gm, m, o);
    offm[i] = o;
  }
  for (int i = tid; i < BN; i += TC_THREADS) {
    const long long n = n0 + i;
    long long o = -1;
    if (n < g.N) decomp(g.gn, n, o);
    offn[i] = o;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const int kt0 = g.splitk > 1 ? int(blockIdx.y) * g.kt_per : 0;
  const int kt_n = g.splitk > 1 ? min(g.kt_per, g.ktiles - kt0) : g.ktiles;   // k tiles of this CTA
  bool ok = true;

  if (warp == 0 && lane == 0) {
    // TMA producer
    const uint32_t tx = uint32_t(stage_bytes);
    for (int kt = 0; kt < kt_n && ok; ++kt) {
      const int s = kt % g.stages;
      const uint32_t round = uint32_t(kt / g.stages);
      ok = mbar_wait(&empty[s], (round & 1u) ^ 1u, g.flag);
      if (!ok) break;
      uint8_t* st = base + s * stage_bytes;
      mbar_expect_tx(&full[s], tx);
      const int kx = (kt0 + kt) * (TC_ROWB / (g.bf16 ? 2 : 4));
      tma_load_2d(st, &ta, &full[s], kx, ra);
      tma_load_2d(st + A_BYTES, &tb, &full[s], kx, rb);
      if (g.split) {
        tma_load_2d(st + A_BYTES + B_BYTES, &tal, &full[s], kx, ra);
        tma_load_2d(st + 2 * A_BYTES + B_BYTES, &tbl, &full[s], kx, rb);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: 4 instructions of K = 32 bytes cover one 128-byte tile row
    const uint32_t afmt = g.bf16 ? 1u : 2u;
    const uint32_t idesc = (1u << 4) | (afmt << 7) | (afmt << 10) | (uint32_t(BN >> 3) << 17) |
                           (uint32_t(TC_BM >> 4) << 24);
    for (int kt = 0; kt < kt_n && ok; ++kt) {
      const int s = kt % g.stages;
      const uint32_t round = uint32_t(kt / g.stages);
      ok = mbar_wait(&full[s], round & 1u, g.flag);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint8_t* st = base + s * stage_bytes;
      const uint64_t da = sdesc(st), db = sdesc(st + A_BYTES);
      const uint64_t dal = sdesc(st + A_BYTES + B_BYTES), dbl = sdesc(st + 2 * A_BYTES + B_BYTES);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t o = uint64_t(kk * 2);   // 32 bytes >> 4
        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
        if (g.bf16) {
          mma_f16(tmem, da + o, db + o, idesc, acc);
          if (g.split) {
            mma_f16(tmem, da + o, dbl + o, idesc, 1u);
            mma_f16(tmem, dal + o, db + o, idesc, 1u);
          }
        } else {
          mma_tf32(tmem, da + o, db + o, idesc, acc);
          if (g.split) {
            mma_tf32(tmem, da + o, dbl + o, idesc, 1u);
            mma_tf32(tmem, dal + o, db + o, idesc, 1u);
          }
        }
      }
      mma_commit(&empty[s]);
    }
    mma_commit(&done);
  }
  __syncwarp();
  // Epilogue: every warp waits for the accumulator (bounded), then reads its 32 lanes.
  const bool waited = mbar_wait(&done, 0u, g.flag);
  const bool have = __all_sync(0xffffffffu, waited && ok);   // warp-uniform: tcgen05.ld is .sync.aligned
  __syncwarp();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int row = warp * 32 + lane;
  const long long om = offm[row];
  const float alpha = float(g.alpha);
  auto put = [&](long long o, float v) { put_out(g, pb, o, v); };
  if (have && g.splitk > 1) {
    // raw partial sums, dense [M][N] per (split, problem), written along N
    float* part = g.part + ((long long)blockIdx.y * g.nprob + pb) * g.M * g.N;
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t r[16];
      tmem_ld16(tmem + (uint32_t(warp * 32) << 16) + uint32_t(c0), r);
#pragma unroll
      for (int j = 0; j < 16; ++j) stage_out[warp][lane][j] = __uint_as_float(r[j]);
      __syncwarp();
      const int j = lane & 15;
      const long long n = n0 + c0 + j;
#pragma unroll 4
      for (int i = lane >> 4; i < 32; i += 2) {
        const long long m = m0 + warp * 32 + i;
        if (m < g.M && n < g.N) part[m * g.N + n] = stage_out[warp][i][j];
      }
      __syncwarp();
    }
  } else if (have) {
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t r[16];
      tmem_ld16(tmem + (uint32_t(warp * 32) << 16) + uint32_t(c0), r);
      if (!g.cols_fast) {
        // one row per lane: coalesced when consecutive rows are adjacent in C
        if (om < 0) continue;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const long long on = offn[c0 + j];
          if (on >= 0) put(om + on, __uint_as_float(r[j]) * alpha);
        }
      } else {
        // through shared memory: 16 lanes per row along the columns
#pragma unroll
        for (int j = 0; j < 16; ++j) stage_out[warp][lane][j] = __uint_as_float(r[j]);
        __syncwarp();
        const int j = lane & 15;
        const long long on = offn[c0 + j];
#pragma unroll 4
        for (int i = lane >> 4; i < 32; i += 2) {
          const long long omi = offm[warp * 32 + i];
          if (omi >= 0 && on >= 0) put(omi + on, stage_out[warp][i][j] * alpha);
        }
        __syncwarp();
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    const uint32_t ncols = BN < 32 ? 32 : BN;
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Persistent form (no split-K): one CTA per SM walks the output tiles t =
// blockIdx.x, blockIdx.x + gridDim.x, ...  Warp 8 (one thread) streams the
// operand tiles through the smem ring with TMA, warp 9 (one thread) issues the
// MMAs into one of two TMEM accumulators, and warps 0-7 drain the other one
// (tcgen05.ld, then the same stores as k_gemm_tc) -- warp w reads TMEM lanes
// 32*(w%4).. and the columns of half w/4 -- so a tile's epilogue runs while
// the next tile is loaded and multiplied.  Every wait is bounded.
constexpr int TCP_THREADS = 320;
constexpr int TCP_EPI = 8;   // epilogue warps

template <int BN>
__global__ void __launch_bounds__(TCP_THREADS) k_gemm_tc_persist(const __grid_constant__ CUtensorMap ta,
                                                                 const __grid_constant__ CUtensorMap tb,
                                                                 const __grid_constant__ CUtensorMap tal,
                                                                 const __grid_constant__ CUtensorMap tbl,
                                                                 const TcArgs g) {
  constexpr int A_BYTES = TC_BM * TC_ROWB;
  constexpr int B_BYTES = BN * TC_ROWB;
  constexpr int NCOL = BN < 32 ? 32 : BN;   // TMEM columns of one accumulator
  extern __shared__ __align__(1024) uint8_t dsm[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~uintptr_t(1023));
  const int stage_bytes = g.split ? 2 * (A_BYTES + B_BYTES) : (A_BYTES + B_BYTES);
  __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES], tfull[2], tempty[2], drain;
  __shared__ uint32_t tmem_base;
  __shared__ long long offm[TC_BM], offn[BN];
  __shared__ float stage_out[TCP_EPI][32][17];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long tiles_n = (g.N + BN - 1) / BN;
  const long long tiles = ((g.M + TC_BM - 1) / TC_BM) * tiles_n;
  const long long total = tiles * g.nprob;
  if (tid == 0) {
    for (int s = 0; s < g.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], TCP_EPI);
    }
    mbar_init(&drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(2 * NCOL));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp == TCP_EPI && lane == 0) {
    // TMA producer, running ahead across tiles
    bool ok = true;
    int it = 0;
    for (long long t = blockIdx.x; t < total && ok; t += gridDim.x) {
      const int pb = int(t / tiles);
      const long long tt = t % tiles;
      const int ra = int(pb * g.pad_m + (tt / tiles_n) * TC_BM), rb = int(pb * g.pad_n + (tt % tiles_n) * BN);
      for (int kt = 0; kt < g.ktiles; ++kt, ++it) {
        const int s = it % g.stages;
        const uint32_t round = uint32_t(it / g.stages);
        ok = mbar_wait(&empty[s], (round & 1u) ^ 1u, g.flag);
        if (!ok) break;
        uint8_t* st = base + s * stage_bytes;
        mbar_expect_tx(&full[s], uint32_t(stage_bytes));
        const int kx = kt * (TC_ROWB / (g.bf16 ? 2 : 4));
        tma_load_2d(st, &ta, &full[s], kx, ra);
        tma_load_2d(st + A_BYTES, &tb, &full[s], kx, rb);
        if (g.split) {
          tma_load_2d(st + A_BYTES + B_BYTES, &tal, &full[s], kx, ra);
          tma_load_2d(st + 2 * A_BYTES + B_BYTES, &tbl, &full[s], kx, rb);
        }
      }
    }
    // no copy of ours may still be landing in shared memory when the CTA leaves:
    // wait (bounded) for the last round issued into every slot
    for (int j = it - 1; j >= 0 && j >= it - g.stages; --j)
      mbar_wait(&full[j % g.stages], uint32_t(j / g.stages) & 1u, g.flag);
  } else if (warp == TCP_EPI + 1 && lane == 0) {
    // MMA issuer: tile i accumulates in TMEM buffer i % 2
    const uint32_t afmt = g.bf16 ? 1u : 2u;
    const uint32_t idesc = (1u << 4) | (afmt << 7) | (afmt << 10) | (uint32_t(BN >> 3) << 17) |
                           (uint32_t(TC_BM >> 4) << 24);
    bool ok = true;
    int it = 0, i = 0;
    for (long long t = blockIdx.x; t < total && ok; t += gridDim.x, ++i) {
      const int buf = i & 1;
      const uint32_t use = uint32_t(i >> 1);
      ok = mbar_wait(&tempty[buf], (use & 1u) ^ 1u, g.flag);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t acc_t = tmem + uint32_t(buf * NCOL);
      for (int kt = 0; kt < g.ktiles; ++kt, ++it) {
        const int s = it % g.stages;
        const uint32_t round = uint32_t(it / g.stages);
        ok = mbar_wait(&full[s], round & 1u, g.flag);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint8_t* st = base + s * stage_bytes;
        const uint64_t da = sdesc(st), db = sdesc(st + A_BYTES);
        const uint64_t dal = sdesc(st + A_BYTES + B_BYTES), dbl = sdesc(st + 2 * A_BYTES + B_BYTES);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t o = uint64_t(kk * 2);
          const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
          if (g.bf16) {
            mma_f16(acc_t, da + o, db + o, idesc, acc);
            if (g.split) {
              mma_f16(acc_t, da + o, dbl + o, idesc, 1u);
              mma_f16(acc_t, dal + o, db + o, idesc, 1u);
            }
          } else {
            mma_tf32(acc_t, da + o, db + o, idesc, acc);
            if (g.split) {
              mma_tf32(acc_t, da + o, dbl + o, idesc, 1u);
              mma_tf32(acc_t, dal + o, db + o, idesc, 1u);
            }
          }
        }
        mma_commit(&empty[s]);
      }
      if (ok) mma_commit(&tfull[buf]);
    }
    // every MMA issued here has finished before TMEM is released (bounded wait)
    mma_commit(&drain);
    mbar_wait(&drain, 0u, g.flag);
  } else if (warp < TCP_EPI) {
    // epilogue: drain the accumulator of tile i while tile i+1 is computed.
    // The eight warps run the same number of iterations and reach both named
    // barriers in every one of them; a warp whose wait ran out (the status word
    // is set) only stops doing work, so no warp is left waiting at a barrier.
    const float alpha = float(g.alpha);
    const int quarter = warp & 3, half = warp >> 2;
    const int cbeg = BN >= 32 ? half * (BN / 2) : (half ? BN : 0), cend = BN >= 32 ? cbeg + BN / 2 : (half ? BN : BN);
    bool dead = false;
    int i = 0;
    for (long long t = blockIdx.x; t < total; t += gridDim.x, ++i) {
      const int buf = i & 1;
      const uint32_t use = uint32_t(i >> 1);
      const int pb = int(t / tiles);
      const long long tt = t % tiles;
      const long long m0 = (tt / tiles_n) * TC_BM, n0 = (tt % tiles_n) * BN;
      asm volatile("bar.sync 1, 256;" ::: "memory");   // the previous tile's offsets are no longer read
      if (tid < TC_BM) {
        const long long m = m0 + tid;
        long long o = -1;
        if (m < g.M) decomp(g.gm, m, o);
        offm[tid] = o;
      }
      for (int c = tid - TC_BM; c >= 0 && c < BN; c += 128) {
        const long long n = n0 + c;
        long long o = -1;
        if (n < g.N) decomp(g.gn, n, o);
        offn[c] = o;
      }
      asm volatile("bar.sync 1, 256;" ::: "memory");
      if (dead) continue;
      const bool waited = mbar_wait(&tfull[buf], use & 1u, g.flag);
      if (!__all_sync(0xffffffffu, waited)) {
        dead = true;
        continue;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int row = quarter * 32 + lane;
      const long long om = offm[row];
      const uint32_t acc_t = tmem + uint32_t(buf * NCOL) + (uint32_t(quarter * 32) << 16);
      for (int c0 = cbeg; c0 < cend; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(acc_t + uint32_t(c0), r);
        if (!g.cols_fast) {
          if (om < 0) continue;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const long long on = offn[c0 + j];
            if (on >= 0) put_out(g, pb, om + on, __uint_as_float(r[j]) * alpha);
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) stage_out[warp][lane][j] = __uint_as_float(r[j]);
          __syncwarp();
          const int j = lane & 15;
          const long long on = offn[c0 + j];
#pragma unroll 4
          for (int q = lane >> 4; q < 32; q += 2) {
            const long long omi = offm[quarter * 32 + q];
            if (omi >= 0 && on >= 0) put_out(g, pb, omi + on, stage_out[warp][q][j] * alpha);
          }
          __syncwarp();
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * NCOL));
  }
}

// Split-K: out[p][m, n] = alpha * sum_s part[s][p][m][n] (fixed order), through
// the output offset groups.
__global__ void k_tc_splitk_reduce(const TcArgs g) {
  const long long MN = g.M * g.N, total = (long long)g.nprob * MN;
  const float alpha = float(g.alpha);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int pb = int(t / MN);
    const long long mn = t - pb * MN, m = mn / g.N, n = mn - m * g.N;
    float v = 0.f;
    for (int sp = 0; sp < g.splitk; ++sp) v += g.part[((long long)sp * g.nprob + pb) * MN + mn];
    v *= alpha;
    long long om, on;
    decomp(g.gm, m, om);
    decomp(g.gn, n, on);
    put_out(g, pb, om + on, v);
  }
}

// Gather-copy into a dense [rows][ld] operand: element (r, k) of the output is
// src[sum(idx_i * stride_i)] with r, k decomposed over the row / K groups.
// Rounds to TF32 (or converts to BF16); `lo` receives the rounded residual.
// Tiled transpose: each CTA moves a 64 x 64 (row, k) tile through shared
// memory, decomposing its 64 row and 64 k offsets once; reads run along
// whichever group holds the source's unit stride (rows_fast), writes run along
// k, so both sides are coalesced whatever the permutation.
struct PackArgs {
  TP src;            // per problem
  int src_f64;
  int rows_fast;     // 1: consecutive rows are closer in src than consecutive k
  Grp gr, gk;        // strides into src
  long long rows, K, ld, pad;   // pad: packed rows per problem
  void* hi;
  void* lo;
  int bf16;
};

// 64 x 64 (row, k) tiles, 256 threads, 16 elements per thread: the offsets
// of a tile's 64 rows and 64 k are decomposed once (128 threads), then every
// thread issues all 16 of its loads before it stores, so each warp keeps 16
// coalesced loads in flight.
constexpr int PK_T = 64;

// hi = v rounded to the operand type; lo = the rounded residual.  For FP32
// sources everything stays in FP32 (v - tf32(v) is exact there): the FP64
// pipe of GB300 is ~1/64 of FP32, so FP64 arithmetic here would bound the copy.
__device__ __forceinline__ void split_store(float v, const PackArgs& p, long long d) {
  if (p.bf16) {
    const __nv_bfloat16 h = __float2bfloat16(v);
    static_cast<__nv_bfloat16*>(p.hi)[d] = h;
    if (p.lo) static_cast<__nv_bfloat16*>(p.lo)[d] = __float2bfloat16(v - __bfloat162float(h));
  } else {
    const float h = round_tf32(v);
    static_cast<float*>(p.hi)[d] = h;
    if (p.lo) static_cast<float*>(p.lo)[d] = round_tf32(v - h);
  }
}
__device__ __forceinline__ void split_store(double v, const PackArgs& p, long long d) {
  if (p.bf16) {
    const __nv_bfloat16 h = __double2bfloat16(v);
    static_cast<__nv_bfloat16*>(p.hi)[d] = h;
    if (p.lo) static_cast<__nv_bfloat16*>(p.lo)[d] = __double2bfloat16(v - double(__bfloat162float(h)));
  } else {
    const float h = round_tf32(float(v));
    static_cast<float*>(p.hi)[d] = h;
    if (p.lo) static_cast<float*>(p.lo)[d] = round_tf32(float(v - double(h)));
  }
}

// Grid = (row tiles x k tiles, problems), 256 threads; T = source element type.
template <typename T>
__global__ void __launch_bounds__(256) k_pack(const PackArgs p) {
  __shared__ T tile[PK_T][PK_T + 1];   // [k][row]
  __shared__ long long ro[PK_T], ko[PK_T];
  const int pb = blockIdx.y;
  const long long ktiles = (p.K + PK_T - 1) / PK_T;
  const long long r0 = (blockIdx.x / ktiles) * PK_T, k0 = (blockIdx.x % ktiles) * PK_T;
  const int tid = threadIdx.x, tx = tid & (PK_T - 1), ty = tid / PK_T;   // ty in 0..3
  if (tid < PK_T) {
    long long o = -1;
    if (r0 + tid < p.rows) decomp(p.gr, r0 + tid, o);
    ro[tid] = o;
  } else if (tid < 2 * PK_T) {
    long long o = -1;
    if (k0 + tid - PK_T < p.K) decomp(p.gk, k0 + tid - PK_T, o);
    ko[tid - PK_T] = o;
  }
  __syncthreads();
  const T* src = static_cast<const T*>(p.src.p[pb]);
  constexpr int NQ = PK_T / 4;   // 16 elements per thread
  T v[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int a = ty + 4 * q;
    const int r = p.rows_fast ? tx : a, k = p.rows_fast ? a : tx;
    const long long orr = ro[r], okk = ko[k];
    v[q] = (orr >= 0 && okk >= 0) ? src[orr + okk] : T(0);
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int a = ty + 4 * q;
    const int r = p.rows_fast ? tx : a, k = p.rows_fast ? a : tx;
    tile[k][r] = v[q];
  }
  __syncthreads();
#pragma unroll 4
  for (int q = 0; q < NQ; ++q) {
    const int r = ty + 4 * q, k = tx;
    if (ro[r] < 0 || ko[k] < 0) continue;
    split_store(tile[k][r], p, (pb * p.pad + r0 + r) * p.ld + k0 + k);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static std::mutex mu;
  static EncodeFn fn = nullptr;
  std::lock_guard<std::mutex> g(mu);
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    PEPS_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    PEPS_REQUIRE(p != nullptr && q == cudaDriverEntryPointSuccess, "cuTensorMapEncodeTiled unavailable");
    fn = reinterpret_cast<EncodeFn>(p);
  }
  return fn;
}

// 2D map of a dense [rows][ld] operand, box = 128 bytes of K x box_rows rows.
CUtensorMap make_map(const void* ptr, long long rows, long long K, long long ld, int bf16, int box_rows) {
  CUtensorMap m;
  std::memset(&m, 0, sizeof(m));
  const int esz = bf16 ? 2 : 4;
  PEPS_REQUIRE((reinterpret_cast<uintptr_t>(ptr) & 15) == 0, "TMA operand not 16-byte aligned");
  PEPS_REQUIRE((ld * esz) % 16 == 0, "TMA row stride not a multiple of 16 bytes");
  cuuint64_t dims[2] = {cuuint64_t(K), cuuint64_t(rows)};
  cuuint64_t strides[1] = {cuuint64_t(ld * esz)};
  cuuint32_t box[2] = {cuuint32_t(TC_ROWB / esz), cuuint32_t(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(&m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                           const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  PEPS_REQUIRE(r == CUDA_SUCCESS, "cuTensorMapEncodeTiled failed: " + std::to_string(int(r)));
  return m;
}

struct Parsed {
  std::string a, b, c;
};

Parsed parse(const char* spec) {
  std::string s(spec);
  auto comma = s.find(','), arrow = s.find("->");
  PEPS_REQUIRE(comma != std::string::npos && arrow != std::string::npos, std::string("bad spec ") + spec);
  return {s.substr(0, comma), s.substr(comma + 1, arrow - comma - 1), s.substr(arrow + 2)};
}

std::vector<long long> strides_of(const Dims& d) {
  std::vector<long long> s(d.size());
  long long acc = 1;
  for (int i = int(d.size()) - 1; i >= 0; --i) {
    s[i] = acc;
    acc *= d[i];
  }
  return s;
}

void push(Grp& g, int dim, long long s) {
  PEPS_REQUIRE(g.n < MAXG, "too many indices in one group");
  g.dim[g.n] = dim;
  g.s[g.n] = s;
  g.n++;
}

long long prod(const Grp& g) {
  long long n = 1;
  for (int i = 0; i < g.n; ++i) n *= g.dim[i];
  return n;
}

struct Operand {
  void* hi = nullptr;
  void* lo = nullptr;
  long long rows = 0, K = 0, ld = 0;
};

// Pack one operand of each of np problems into [np * pad][ld] (rows over
// `rowletters`, K over `kletters`; problem p at rows p * pad ..).
Operand pack(Ctx& cx, const TP& src, int np, long long pad, int src_f64, const std::string& letters,
             const Dims& dims, const std::string& rowletters, const std::string& kletters, int bf16, int split,
             double* mem) {
  auto st = strides_of(dims);
  PackArgs p;
  std::memset(static_cast<void*>(&p), 0, sizeof(p));
  for (char ch : rowletters) {
    auto i = letters.find(ch);
    push(p.gr, dims[i], st[i]);
  }
  for (char ch : kletters) {
    auto i = letters.find(ch);
    push(p.gk, dims[i], st[i]);
  }
  Operand o;
  o.rows = prod(p.gr);
  o.K = prod(p.gk);
  const int align = bf16 ? 8 : 4;
  o.ld = (o.K + align - 1) / align * align;
  PEPS_REQUIRE(pad >= o.rows, "internal: pack padding");
  const size_t bytes = size_t(np) * size_t(pad) * o.ld * (bf16 ? 2 : 4);
  const size_t words = (bytes + 255) / 256 * 32;   // doubles, 256-byte aligned
  o.hi = mem;
  o.lo = split ? static_cast<void*>(mem + words) : nullptr;
  p.src = src.all(np);
  p.src_f64 = src_f64;
  p.rows = o.rows;
  p.K = o.K;
  p.ld = o.ld;
  p.pad = pad;
  p.hi = o.hi;
  p.lo = o.lo;
  p.bf16 = bf16;
  // read along whichever group holds the smaller innermost stride
  auto inner = [](const Grp& g) {
    long long m = 1LL << 62;
    for (int i = 0; i < g.n; ++i)
      if (g.dim[i] > 1) m = std::min(m, g.s[i]);
    return m;
  };
  p.rows_fast = inner(p.gr) < inner(p.gk) ? 1 : 0;
  const long long tiles = ((o.rows + PK_T - 1) / PK_T) * ((o.K + PK_T - 1) / PK_T);
  PEPS_REQUIRE(tiles < (1LL << 31), "operand too large to pack");
  const double moved = double(np) * double(o.rows) * double(o.K) *
                       ((src_f64 ? 8.0 : 4.0) + (split ? 2.0 : 1.0) * (bf16 ? 2.0 : 4.0));
  Launch L(K_PACK, cx.st, 0, moved);
  if (src_f64)
    k_pack<double><<<dim3(unsigned(tiles), np), 256, 0, cx.st>>>(p);
  else
    k_pack<float><<<dim3(unsigned(tiles), np), 256, 0, cx.st>>>(p);
  PEPS_CHECK_LAUNCH();
  return o;
}

size_t pack_words(long long rows, long long K, int bf16, int split) {
  const int align = bf16 ? 8 : 4;
  const long long ld = (K + align - 1) / align * align;
  const size_t bytes = size_t(rows) * ld * (bf16 ? 2 : 4);
  const size_t words = (bytes + 255) / 256 * 32;
  return split ? 2 * words : words;
}

template <int BN>
void launch_tc(Ctx& cx, const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& tal,
               const CUtensorMap& tbl, TcArgs g, long long tiles) {
  const int a_bytes = TC_BM * TC_ROWB, b_bytes = BN * TC_ROWB;
  const int stage = g.split ? 2 * (a_bytes + b_bytes) : (a_bytes + b_bytes);
  const int budget = 200 * 1024;
  g.stages = std::max(1, std::min({TC_STAGES, (budget - 1024) / stage, g.splitk > 1 ? g.kt_per : g.ktiles}));
  const size_t smem = size_t(stage) * g.stages + 1024;
  static std::once_flag once;
  static int nsm = 0;
  static bool persist = true;   // PEPS_TC_PERSIST=0 keeps every GEMM on the one-tile kernel
  std::call_once(once, [] {
    PEPS_CUDA(cudaFuncSetAttribute(k_gemm_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    PEPS_CUDA(cudaFuncSetAttribute(k_gemm_tc_persist<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    int dev = 0;
    PEPS_CUDA(cudaGetDevice(&dev));
    PEPS_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (const char* e = std::getenv("PEPS_TC_PERSIST")) persist = std::atoi(e) != 0;
  });
  if (!persist || g.splitk > 1 || tiles <= nsm) {
    // split-K partials, or no more tiles than SMs: one tile per CTA
    k_gemm_tc<BN><<<dim3(unsigned(tiles), unsigned(std::max(1, g.splitk))), TC_THREADS, smem, cx.st>>>(ta, tb, tal,
                                                                                                        tbl, g);
  } else {
    // the ring holds at least two stages so the next tile's operands stream in
    g.stages = std::max(1, std::min(TC_STAGES, (budget - 1024) / stage));
    const size_t psmem = size_t(stage) * g.stages + 1024;
    k_gemm_tc_persist<BN><<<unsigned(nsm), TCP_THREADS, psmem, cx.st>>>(ta, tb, tal, tbl, g);
  }
  PEPS_CHECK_LAUNCH();
}

}  // namespace

int tc_available() {
  static int ok = -1;
  if (ok < 0) {
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    ok = (major == 10 && minor == 3) ? 1 : 0;
  }
  return ok;
}

// Operand A of `spec` as ein_tc lays it out: M rows over the output letters
// taken from A (in the output's order), K over A's summed letters (in A's
// order), rows padded to the tile height per problem, K padded to 16 bytes.
struct LayoutA {
  std::string a;            // the contraction's operand-A letters, in operand order
  std::string rows, ks;
  std::vector<long long> rdim, kdim;
  long long M = 1, K = 1, pad = 0, ld = 0;
  size_t words = 0;   // doubles of the hi array; the lo array follows
};

LayoutA layout_a(const char* spec, const Dims& ad, const Dims& bd, int np, int prec) {
  const Parsed p = parse(spec);
  (void)bd;
  LayoutA L;
  L.a = p.a;
  for (char ch : p.c)
    if (p.a.find(ch) != std::string::npos) {
      L.rows += ch;
      L.rdim.push_back(ad[p.a.find(ch)]);
      L.M *= ad[p.a.find(ch)];
    }
  for (char ch : p.a)
    if (p.c.find(ch) == std::string::npos) {
      L.ks += ch;
      L.kdim.push_back(ad[p.a.find(ch)]);
      L.K *= ad[p.a.find(ch)];
    }
  const int bf16 = (prec == PEPS_PREC_BF16 || prec == PEPS_PREC_BF16X3) ? 1 : 0;
  const int align = bf16 ? 8 : 4;
  L.pad = (L.M + TC_BM - 1) / TC_BM * TC_BM;
  L.ld = (L.K + align - 1) / align * align;
  L.words = pack_words(np * L.pad, L.K, bf16, 0);
  return L;
}

size_t tc_operand_words(const char* spec, const Dims& ad, const Dims& bd, int np, int prec) {
  const int split = (prec == PEPS_PREC_TF32X3 || prec == PEPS_PREC_BF16X3) ? 1 : 0;
  return (split ? 2 : 1) * layout_a(spec, ad, bd, np, prec).words;
}

void ein_tc(Ctx& cx, const char* spec, const TP& A, int a_f64, const Dims& ad, const TP& B, int b_f64,
            const Dims& bd, const TP& C, int c_f64, int prec, double alpha, const TP& Clo, PackCache* bcache,
            const TcChain* chain) {
  PEPS_REQUIRE(tc_available(), "tensor-core path needs an sm_103 device");
  const bool to_next = chain && chain->next;
  const TcOperand* a_pre = chain ? chain->a_pre : nullptr;
  int np = to_next ? problems({&A, &B}) : problems({&A, &B, &C, &Clo});
  if (a_pre) {
    PEPS_REQUIRE(np == 1 || np == a_pre->np, "internal: pre-packed operand for another problem count");
    np = a_pre->np;
  }
  PEPS_REQUIRE(!B.null() && (a_pre || !A.null()) && (to_next || (C.n == np && (Clo.null() || Clo.n == np))),
               "internal: contraction operands");
  const Parsed p = parse(spec);
  const Dims cd = ein_dims(spec, ad, bd);
  const auto sc = strides_of(cd);
  const int bf16 = (prec == PEPS_PREC_BF16 || prec == PEPS_PREC_BF16X3) ? 1 : 0;
  const int split = (prec == PEPS_PREC_TF32X3 || prec == PEPS_PREC_BF16X3) ? 1 : 0;
  // Output strides: C's own (row-major over the output letters), or those of
  // operand A of the next contraction.
  // (output index i is index i of the next contraction's operand A, whose
  // letters may be named differently there)
  std::vector<long long> ostr(sc.begin(), sc.end());
  LayoutA nx;
  if (to_next) {
    nx = layout_a(chain->next, cd, chain->next_bd, np, prec);
    PEPS_REQUIRE(nx.a.size() == p.c.size() && nx.rows.size() + nx.ks.size() == p.c.size(),
                 "internal: chained operand letters");
    for (size_t i = 0; i < p.c.size(); ++i) {
      const char ch = nx.a[i];
      long long st = 1;
      auto r = nx.rows.find(ch), k = nx.ks.find(ch);
      if (r != std::string::npos) {
        st = nx.ld;
        for (size_t j = r + 1; j < nx.rows.size(); ++j) st *= nx.rdim[j];
        PEPS_REQUIRE(nx.rdim[r] == cd[i], "internal: chained operand dims");
      } else {
        PEPS_REQUIRE(k != std::string::npos && nx.kdim[k] == cd[i], "internal: chained operand letters");
        for (size_t j = k + 1; j < nx.ks.size(); ++j) st *= nx.kdim[j];
      }
      ostr[i] = st;
    }
    PEPS_REQUIRE((split ? 2 : 1) * nx.words <= chain->next_cap, "internal: chained operand buffer too small");
  }
  std::string mL, nL, kL;
  TcArgs g;
  std::memset(static_cast<void*>(&g), 0, sizeof(g));
  for (size_t i = 0; i < p.c.size(); ++i) {
    const char ch = p.c[i];
    const bool inA = p.a.find(ch) != std::string::npos, inB = p.b.find(ch) != std::string::npos;
    PEPS_REQUIRE(!(inA && inB), std::string("batch index not supported on the tensor-core path: ") + spec);
    if (inA) {
      mL += ch;
      push(g.gm, cd[i], ostr[i]);
    } else {
      nL += ch;
      push(g.gn, cd[i], ostr[i]);
    }
  }
  for (char ch : p.a)
    if (p.c.find(ch) == std::string::npos) {
      PEPS_REQUIRE(p.b.find(ch) != std::string::npos, std::string("unsupported one-sided sum: ") + spec);
      kL += ch;
    }
  long long M = 1, N = 1, K = 1;
  for (char ch : mL) M *= ad[p.a.find(ch)];
  for (char ch : nL) N *= bd[p.b.find(ch)];
  for (char ch : kL) K *= ad[p.a.find(ch)];
  if (M == 0 || N == 0) return;
  int BN = 16;
  while (BN < N && BN < 128) BN *= 2;
  const long long pad_m = (M + TC_BM - 1) / TC_BM * TC_BM, pad_n = (N + BN - 1) / BN * BN;
  if (a_pre)
    PEPS_REQUIRE(a_pre->pad == pad_m && a_pre->ld == (K + (bf16 ? 8 : 4) - 1) / (bf16 ? 8 : 4) * (bf16 ? 8 : 4),
                 "internal: pre-packed operand layout");
  const size_t wa = a_pre ? 0 : pack_words(np * pad_m, K, bf16, split);
  const size_t wb_need = pack_words(np * pad_n, K, bf16, split);
  // a cached B operand: packed once into the cache's memory
  PackCache::Entry* cached = nullptr;
  bool fresh = false;
  if (bcache) {
    std::string key = std::string(spec) + '|' + std::to_string(np) + '|' + std::to_string(bf16) +
                      std::to_string(split) + '|' + std::to_string(BN);
    for (int b = 0; b < np; ++b) key += '|' + std::to_string(reinterpret_cast<uintptr_t>(B.v(b)));
    auto it = bcache->entries.find(key);
    if (it == bcache->entries.end()) {
      double* m = bcache->mem->dalloc(wb_need);
      const size_t words = wb_need / (split ? 2 : 1);
      it = bcache->entries.emplace(key, PackCache::Entry{m, split ? static_cast<void*>(m + words) : nullptr, 0}).first;
      fresh = true;
    }
    cached = &it->second;
  }
  const size_t wb = cached ? 0 : wb_need;
  const long long tiles = ((M + TC_BM - 1) / TC_BM) * ((N + BN - 1) / BN) * np;
  PEPS_REQUIRE(tiles < (1LL << 31), "too many tiles");
  g.ktiles = int((K + (TC_ROWB / (bf16 ? 2 : 4)) - 1) / (TC_ROWB / (bf16 ? 2 : 4)));
  // Split K when the output tiles would leave most SMs idle: each split runs
  // at least two k tiles; partials are reduced in a fixed order.
  g.splitk = 1;
  g.kt_per = g.ktiles;
  if (tiles < 152 && g.ktiles >= 4) {
    const long long want = std::min<long long>((2 * 152 + tiles - 1) / tiles, g.ktiles / 2);
    if (want > 1) {
      g.kt_per = int((g.ktiles + want - 1) / want);
      g.splitk = int((g.ktiles + g.kt_per - 1) / g.kt_per);
    }
  }
  const size_t wp = g.splitk > 1 ? (size_t(g.splitk) * np * M * N + 1) / 2 + 64 : 0;
  double* mem = cx.scratch(wa + wb + wp);   // one reservation: operands, then split partials
  if (g.splitk > 1) g.part = reinterpret_cast<float*>(mem + wa + wb);
  Operand oa;
  if (a_pre) {
    oa.hi = a_pre->hi;
    oa.lo = a_pre->lo;
    oa.rows = M;
    oa.K = K;
    oa.ld = a_pre->ld;
  } else {
    oa = pack(cx, A, np, pad_m, a_f64, p.a, ad, mL, kL, bf16, split, mem);
  }
  Operand ob;
  if (!cached || fresh) {
    ob = pack(cx, B, np, pad_n, b_f64, p.b, bd, nL, kL, bf16, split,
              cached ? static_cast<double*>(cached->hi) : mem + wa);
    if (cached) cached->ld = ob.ld;
  } else {
    ob.hi = cached->hi;
    ob.lo = cached->lo;
    ob.rows = N;
    ob.K = K;
    ob.ld = cached->ld;
  }
  PEPS_REQUIRE(np * pad_m < (1LL << 31) && np * pad_n < (1LL << 31), "operand too large for one launch");
  const CUtensorMap ta = make_map(oa.hi, np * pad_m, K, oa.ld, bf16, TC_BM);
  const CUtensorMap tb = make_map(ob.hi, np * pad_n, K, ob.ld, bf16, BN);
  const CUtensorMap tal = split ? make_map(oa.lo, np * pad_m, K, oa.ld, bf16, TC_BM) : ta;
  const CUtensorMap tbl = split ? make_map(ob.lo, np * pad_n, K, ob.ld, bf16, BN) : tb;
  g.M = M;
  g.N = N;
  g.K = K;
  g.split = split;
  g.bf16 = bf16;
  if (to_next) {
    const size_t esz = bf16 ? 2 : 4;
    char* hi = reinterpret_cast<char*>(chain->next_mem);
    char* lo = split ? hi + nx.words * sizeof(double) : nullptr;
    TP ch, cl;
    ch.n = np;
    cl.n = split ? np : 0;
    for (int b = 0; b < np; ++b) {
      ch.p[b] = hi + size_t(b) * nx.pad * nx.ld * esz;
      if (split) cl.p[b] = lo + size_t(b) * nx.pad * nx.ld * esz;
    }
    g.C = ch;
    g.Clo = cl;
    g.out_f64 = 0;
    g.out_lo = split;
    g.out_tc = bf16 ? 2 : 1;
    if (chain->next_out) {
      TcOperand& o = *chain->next_out;
      o.hi = hi;
      o.lo = lo;
      o.ld = nx.ld;
      o.pad = nx.pad;
      o.np = np;
    }
  } else {
    g.out_f64 = c_f64;
    g.out_lo = (!Clo.null() && !c_f64) ? 1 : 0;
    g.C = C.all(np);
    g.Clo = Clo.all(np);
  }
  {
    // Epilogue store pattern: one row per lane (a warp stores 32 rows of one
    // column) or 16 lanes per row through shared memory (2 rows x 16 columns).
    // Take the one whose warp store touches fewer 32-byte sectors in the
    // first tile; on a tie, the one along the smaller innermost stride.
    auto inner = [](const Grp& q) {
      long long m = 1LL << 62;
      for (int i = 0; i < q.n; ++i)
        if (q.dim[i] > 1) m = std::min(m, q.s[i]);
      return m;
    };
    auto offset = [](const Grp& q, long long idx) {
      long long o = 0;
      for (int i = q.n - 1; i >= 0; --i) {
        o += (idx % q.dim[i]) * q.s[i];
        idx /= q.dim[i];
      }
      return o;
    };
    const int esz = g.out_f64 ? 8 : (g.out_tc == 2 ? 2 : 4);
    auto sectors = [&](bool cols) {
      std::vector<long long> v;
      const int ri = cols ? 2 : 32, cj = cols ? 16 : 1;
      for (int i = 0; i < ri && i < M; ++i)
        for (int j = 0; j < cj && j < N; ++j) v.push_back((offset(g.gm, i) + offset(g.gn, j)) * esz / 32);
      std::sort(v.begin(), v.end());
      return std::unique(v.begin(), v.end()) - v.begin();
    };
    const long long sc_cols = sectors(true), sc_rows = sectors(false);
    g.cols_fast = sc_cols != sc_rows ? (sc_cols < sc_rows ? 1 : 0) : (inner(g.gn) < inner(g.gm) ? 1 : 0);
  }
  g.nprob = np;
  g.pad_m = pad_m;
  g.pad_n = pad_n;
  g.alpha = alpha;
  g.flag = cx.flag;
  const double flops = 2.0 * double(M) * double(N) * double(K) * np;
  // algorithmic bytes: both packed operands read once, the output written once
  // (as the next contraction's packed operand, FP64, or FP32 with its residual)
  const double in_b = (bf16 ? 2.0 : 4.0) * (split ? 2.0 : 1.0);
  const double out_b = to_next ? in_b : (g.out_f64 ? 8.0 : (g.out_lo ? 8.0 : 4.0));
  const double bytes = double(np) * (double(M) * K * in_b + double(N) * K * in_b + double(M) * N * out_b);
  Launch L(K_GEMM_TC, cx.st, flops, bytes);
  switch (BN) {
    case 16: launch_tc<16>(cx, ta, tb, tal, tbl, g, tiles); break;
    case 32: launch_tc<32>(cx, ta, tb, tal, tbl, g, tiles); break;
    case 64: launch_tc<64>(cx, ta, tb, tal, tbl, g, tiles); break;
    default: launch_tc<128>(cx, ta, tb, tal, tbl, g, tiles); break;
  }
  if (g.splitk > 1) {
    const long long total = (long long)np * M * N;
    const unsigned blocks = unsigned(std::max<long long>(1, std::min<long long>((total + 255) / 256, 4096)));
    k_tc_splitk_reduce<<<blocks, 256, 0, cx.st>>>(g);
    PEPS_CHECK_LAUNCH();
    L.more();
  }
}

}  // namespace peps
