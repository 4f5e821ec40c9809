// Complex GEMM step on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// C[p][m][n] = sum_k A[mapA(p)][m][k] * B[mapB(p)][k][n] in complex64 is run as
// one real GEMM on interleaved data (the 4M real embedding):
//     C_r[m][j] = sum_i A_r[m][i] * Bt[j][i],  A_r = A viewed as fp32 [M][2K],
//     Bt = the real embedding of B, [2N][2K] K-major (built by k_bprep_tc).
// FP32 accuracy from TF32 tensor cores by the 3xTF32 split
//     A_r Bt ~ A_hi B_hi + A_hi B_lo + A_lo B_hi,
// hi = round-to-tf32, lo = x - hi.  The BF16 engine takes the same three
// products of bf16 hi/lo parts on kind::f16 (~2^-16 relative per product, at
// twice the tensor rate); the FP16 engine takes them of fp16 hi/lo parts of
// the operands scaled by powers of two (fp16 and tf32 both carry 11
// significant bits, so it keeps the 3xTF32 accuracy at the kind::f16 rate;
// the scales, exact, are undone in the epilogue).  Both operands arrive pre-split in global
// memory (A by the split-mode permute, B by k_bprep_tc), so the kernel is a
// plain TMA -> MMA pipeline.
//
// Accumulation: the tensor cores' own FP32 accumulation is not round-to-
// nearest, so a long K loop accumulated in place drifts (the error grows
// linearly with K; see Ootomo and Yokota, "Recovering single precision
// accuracy from Tensor Cores while surpassing the FP32 theoretical peak
// performance", 2022).  The K loop is therefore cut into chunks of K (see
// chunk_bytes), each accumulated from zero in one of two ping-pong TMEM
// buffers (2 x BN <= 512 columns) and folded by eight drain warps into a
// running sum held in their registers with ordinary round-to-nearest FP32
// adds, while the MMAs of the next chunk fill the other buffer.
//
// Roles (320 threads): warps 0-7 drain chunk accumulators into the running sum
// and write the tile out (two warps per TMEM lane quarter, half the columns
// each), warp 8 issues TMA loads, warp 9 owns TMEM and issues the MMAs.  The
// kernel is persistent: one CTA per SM walks 128 x BN tiles of C_r with a
// stride of the grid, its pipeline and chunk counters running on across
// tiles, so the loads and MMAs of the next tile proceed while the drain warps
// write the previous tile out of their registers.
//
// Patterns folded into N: when every pattern shares A (the sparse-state
// batch of one big tensor against many small ones) and 2N is narrower than
// the tile, one tile covers BN / 2N consecutive patterns side by side (each
// pattern's B rows loaded as its own box), so narrow steps still run
// 256-wide MMAs.
//
// Every mbarrier wait is bounded; on timeout the CTA records a status code,
// leaves its loops, waits (again bounded) for its TMA loads and MMAs still in
// flight, frees its TMEM and exits instead of hanging.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "kernels.h"

namespace tn {

namespace tc {

constexpr int BM = 128;
// K per k-block (one pipeline stage), KB bytes of each operand row: 128 (the
// 128-byte swizzle) or 64 (the 64-byte swizzle; stages half the size, twice
// as many in flight, half the MMAs per k-block).
// Choice per instantiation (measured on the 30-qubit plan): 128-byte
// k-blocks for the 16-bit formats up to BN = 128, where the MMAs are short
// and the per-k-block issue cost shows; 64-byte ones for tf32 and for BN = 256,
// where more stages in flight hide the TMA latency.
__host__ __device__ constexpr int kb_bytes(int BN, int FMT) { return (FMT == 0 || BN >= 256) ? 64 : 128; }
// stages that fit 227 KB of shared memory for a 128 x BN tile
__host__ __device__ constexpr int kb_stages(int BN, int KB) {
  return KB == 128 ? (BN <= 16 ? 6 : BN <= 32 ? 5 : BN <= 64 ? 4 : BN <= 128 ? 3 : 2)
                   : (BN <= 64 ? 8 : BN <= 128 ? 6 : 4);
}

template <int KB>
struct KBlock {
  static constexpr int KK = KB / 32;      // MMAs per product per k-block (32 bytes of K each)
};

// Bytes of K per chunk (one fresh TMEM accumulation, then one drain into the
// registers' running sum).  Longer chunks drain less often: on the 30-qubit
// workload the drain of 128-byte chunks held back the MMAs (the dominant
// pair GEMM ran 8 % faster with 256-byte chunks and 11 % with 512-byte ones),
// but each chunk adds more MMA results in the tensor cores' own accumulation.
// Relative error of the 64-slice head against the O1 state vector with 128,
// 256 and 512-byte chunks: FP16x3 1.9e-6, 3.4e-6, 5.8e-6; 3xTF32 2.4e-6,
// 4.0e-6, 7.1e-6; BF16x3 2.02e-5, 2.05e-5, 2.10e-5 (its 8-bit split
// dominates).  So the engines bound at 1e-5 (3xTF32, FP16x3) take 256 bytes
// (64 tf32 or 128 fp16 terms) and BF16x3, bound at 1e-4, takes 512.
__host__ __device__ constexpr int chunk_bytes(int FMT) { return FMT == 1 ? 512 : 256; }
constexpr int kThreads = 320;
constexpr uint32_t kWaitLimit = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\tselp.u32 %0, 1, 0, P;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: returns false (and flags the CTA) if the phase never completes.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  for (uint32_t i = 0; i < kWaitLimit; ++i) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

// Bounded wait that ignores the abort flag: used on the way out, to let
// copies and MMAs already issued finish before the CTA frees its resources.
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < kWaitLimit; ++i)
    if (mbar_try(bar, parity)) return;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

// UMMA shared-memory descriptor: K-major, KB-byte swizzle (128 or 64), 8-row
// groups 8 * KB bytes apart.
template <int KB>
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)((8 * KB) >> 4) << 32;            // stride byte offset
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)(KB == 128 ? 2 : 4) << 61;        // SWIZZLE_128B : SWIZZLE_64B
  return d;
}

// Instruction descriptor: D f32, A/B tf32 (format 2), bf16 (format 1) or fp16
// (format 0), both K-major, M = 128, N = BN.  FMT: 0 tf32, 1 bf16, 2 fp16.
template <int BN, int FMT>
__device__ __forceinline__ uint32_t idesc_mma() {
  const uint32_t f = FMT == 0 ? 2u : (FMT == 1 ? 1u : 0u);
  return (1u << 4) | (f << 7) | (f << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

// One MMA: K = 8 (tf32) or 16 (bf16, fp16), i.e. 32 bytes of each operand row.
template <bool H16>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if (H16)
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

template <int BN, int STAGES, int KB>
struct Layout {
  static constexpr int A_BYTES = BM * KB;              // one 128-row tile, KB bytes of K per row
  static constexpr int B_BYTES = BN * KB;              // one BN-row tile
  static constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;  // A hi, A lo, B hi, B lo
  static constexpr int DATA = STAGES * STAGE;
  static constexpr int TOTAL = DATA + 1024 /*align*/ + 256 /*barriers*/;
  static_assert(TOTAL <= 232448, "shared memory per CTA");
  static_assert(2 * STAGES + 8 <= 32, "barrier area");
  // two chunk buffers of BN fp32 columns (ping-pong), a power of two >= 32
  static constexpr uint32_t TMEM_COLS = 2 * BN < 32 ? 32 : 2 * BN;
};

// Tile order: groups of GROUP_M m-tiles; inside a group n-tiles and (when A is
// shared by every pattern) patterns vary before the next group, so the A rows
// of a group and the B tiles of a wave stay in L2.
constexpr int64_t GROUP_M = 8;

__device__ __forceinline__ void tile_coords(int64_t t, int64_t tilesM, int64_t tilesN, int64_t PC, bool a_shared,
                                            int64_t& pc, int64_t& tm, int64_t& tn) {
  const int64_t P_in = a_shared ? PC : 1;
  int64_t outer = 0;
  if (!a_shared) {
    outer = t / (tilesM * tilesN);
    t -= outer * tilesM * tilesN;
  }
  const int64_t per_full = GROUP_M * tilesN * P_in;
  const int64_t mg = t / per_full;
  int64_t r = t - mg * per_full;
  const int64_t gm = min(GROUP_M, tilesM - mg * GROUP_M);
  const int64_t mi = r % gm;
  r /= gm;
  tn = r % tilesN;
  const int64_t pin = r / tilesN;
  tm = mg * GROUP_M + mi;
  pc = a_shared ? pin : outer;
}

template <int BN, int STAGES, int FMT>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmAhi, const __grid_constant__ CUtensorMap tmAlo,
              const __grid_constant__ CUtensorMap tmBhi, const __grid_constant__ CUtensorMap tmBlo,
              float* __restrict__ C, int64_t M, int64_t N2, int64_t K2, int64_t tilesM, int64_t tilesN, int64_t PC,
              int64_t PCg, int fold, const uint32_t* __restrict__ mapA, const uint32_t* __restrict__ mapB,
              int mapA_mode, int mapB_mode, const unsigned int* scaleA, const unsigned int* scaleB,
              unsigned int* amax_out, unsigned int* status) {
  constexpr int KB = kb_bytes(BN, FMT);
  constexpr int CH = chunk_bytes(FMT) / KB;   // k-blocks per chunk
  using Lay = Layout<BN, STAGES, KB>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + Lay::DATA);
  uint64_t* full = bars;                    // stage loaded   [STAGES]
  uint64_t* empty = bars + STAGES;          // stage consumed [STAGES]
  uint64_t* accf = bars + 2 * STAGES;       // chunk accumulated (MMA -> drain) [2]
  uint64_t* acce = bars + 2 * STAGES + 2;   // chunk drained (drain -> MMA)     [2]
  uint64_t* mma_done = bars + 2 * STAGES + 4;   // every issued MMA complete (before TMEM is freed)
  volatile uint32_t* tmem_slot = (volatile uint32_t*)(bars + 2 * STAGES + 5);
  volatile int* abort_flag = (volatile int*)(bars + 2 * STAGES + 6);
  unsigned int* s_amax = (unsigned int*)(bars + 2 * STAGES + 7);   // CTA maximum of its output tiles

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool a_shared = mapA_mode == 1 && PC > 1;
  const int64_t n_tiles = tilesM * tilesN * PCg;
  const int br = BN / fold;                 // B rows per pattern box (2N when folded)
  constexpr bool H16 = FMT != 0;
  constexpr int BKE = KB / (H16 ? 2 : 4);   // K elements per k-block
  constexpr int KK = KBlock<KB>::KK;
  const int nkb = (int)((K2 + BKE - 1) / BKE);
  const int nch = (nkb + CH - 1) / CH;
  // tile t -> first pattern pc0 of its group, m-tile, n-tile
  auto coords = [&](int64_t t, int64_t& pc0, int64_t& tm, int64_t& tn_) {
    int64_t pg;
    tile_coords(t, tilesM, tilesN, PCg, a_shared, pg, tm, tn_);
    pc0 = pg * fold;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 8);               // one arrive per drain warp
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    *s_amax = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 9) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32((const void*)tmem_slot)),
                 "r"(Lay::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;

  if (warp == 8) {
    if (lane == 0) {
      uint32_t it = 0;          // k-blocks issued by this CTA (all tiles)
      bool ok = true;
      for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        int64_t pc0, tm, tn_;
        coords(t, pc0, tm, tn_);
        const int64_t pa = mapA_mode == 0 ? pc0 : (mapA_mode == 1 ? 0 : (int64_t)mapA[pc0]);
        for (int kb = 0; kb < nkb; ++kb) {
          const int s = (int)(it % STAGES);
          const uint32_t r = it / STAGES;
          if (!mbar_wait(&empty[s], (r & 1) ^ 1, abort_flag)) { ok = false; break; }
          uint8_t* st = smem + s * Lay::STAGE;
          mbar_expect_tx(&full[s], (uint32_t)Lay::STAGE);
          tma_load_3d(st, &tmAhi, &full[s], kb * BKE, (int)(tm * BM), (int)pa);
          tma_load_3d(st + Lay::A_BYTES, &tmAlo, &full[s], kb * BKE, (int)(tm * BM), (int)pa);
          for (int f = 0; f < fold; ++f) {
            // a pattern past the last one loads pattern PC - 1 again: its
            // columns are computed but never stored
            const int64_t pcf = pc0 + f < PC ? pc0 + f : PC - 1;
            const int64_t pb = mapB_mode == 0 ? pcf : (mapB_mode == 1 ? 0 : (int64_t)mapB[pcf]);
            uint8_t* sb = st + 2 * Lay::A_BYTES + f * br * KB;
            tma_load_3d(sb, &tmBhi, &full[s], kb * BKE, (int)(tn_ * br), (int)pb);
            tma_load_3d(sb + Lay::B_BYTES, &tmBlo, &full[s], kb * BKE, (int)(tn_ * br), (int)pb);
          }
          ++it;
        }
      }
      if (!ok) {
        // only the last STAGES issued k-blocks can still be landing
        for (uint32_t j = it > (uint32_t)STAGES ? it - STAGES : 0; j < it; ++j)
          mbar_drain(&full[j % STAGES], (j / STAGES) & 1);
      }
    }
  } else if (warp == 9) {
    if (lane == 0) {
      const uint32_t idesc = idesc_mma<BN, FMT>();
      uint32_t it = 0, cc = 0;   // k-blocks and chunks consumed by this CTA (all tiles)
      bool ok = true, issued = false;
      for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        for (int kb = 0; kb < nkb; ++kb) {
          // chunk cc accumulates in TMEM buffer b = cc & 1 from zero
          const int s = (int)(it % STAGES);
          const uint32_t r = it / STAGES;
          const int b = (int)(cc & 1);
          const uint32_t u = cc >> 1;   // use index of buffer b
          const bool first = kb % CH == 0, last = kb % CH == CH - 1 || kb == nkb - 1;
          if (first && !mbar_wait(&acce[b], (u & 1) ^ 1, abort_flag)) { ok = false; break; }
          if (!mbar_wait(&full[s], r & 1, abort_flag)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t d = tmem + (uint32_t)(b * BN);
          const uint32_t st = smem_u32(smem + s * Lay::STAGE);
          const uint32_t a_hi = st, a_lo = st + Lay::A_BYTES;
          const uint32_t b_hi = st + 2 * Lay::A_BYTES, b_lo = b_hi + Lay::B_BYTES;
          // small correction products first, so that the accumulator is still
          // small while they are added; the hi x hi products come last
#pragma unroll
          for (int kk = 0; kk < KK; ++kk) {
            const uint32_t o = kk * 32;  // one MMA's K = 32 bytes of each operand row
            mma<H16>(d, sdesc<KB>(a_hi + o), sdesc<KB>(b_lo + o), idesc, (first && kk == 0) ? 0u : 1u);
            mma<H16>(d, sdesc<KB>(a_lo + o), sdesc<KB>(b_hi + o), idesc, 1u);
          }
#pragma unroll
          for (int kk = 0; kk < KK; ++kk) {
            const uint32_t o = kk * 32;
            mma<H16>(d, sdesc<KB>(a_hi + o), sdesc<KB>(b_hi + o), idesc, 1u);
          }
          issued = true;
          mma_commit(&empty[s]);
          if (last) {
            mma_commit(&accf[b]);
            ++cc;
          }
          ++it;
        }
      }
      // every issued MMA has completed before TMEM is freed (also on abort)
      if (issued) {
        mma_commit(mma_done);
        mbar_drain(mma_done, 0);
      }
    }
  } else {
    // drain warps 0-7: TMEM lane quarter = warp % 4, column half = warp / 4;
    // each thread keeps the running sum of its row's NCOL columns in registers.
    constexpr int NCOL = BN >= 32 ? BN / 2 : BN;     // columns per warp
    constexpr int NPIECE = NCOL / 16;                  // 16-column TMEM loads
    constexpr int RPMAX = BN >= 256 ? 2 : 4;           // loads in flight per wait
    constexpr int RP = NPIECE < RPMAX ? NPIECE : RPMAX;
    const int q = warp & 3, half = warp >> 2;
    const bool active = BN >= 32 || half == 0;
    const int col0 = BN >= 32 ? half * NCOL : 0;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    // FP16 engine: undo the operands' power-of-two scales (two exact multiplies)
    const float ua = FMT == 2 ? pow2f(-fp16_scale_exp(*scaleA)) : 1.0f;
    const float ub = FMT == 2 ? pow2f(-fp16_scale_exp(*scaleB)) : 1.0f;
    float tmax = 0.0f;
    uint32_t cc = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
      int64_t pc0, tm, tn_;
      coords(t, pc0, tm, tn_);
      float acc[NCOL];
#pragma unroll
      for (int e = 0; e < NCOL; ++e) acc[e] = 0.0f;
      for (int c = 0; c < nch; ++c) {
        const int b = (int)(cc & 1);
        const uint32_t u = cc >> 1;
        ok = mbar_wait(&accf[b], u & 1, abort_flag);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (active) {
#pragma unroll
          for (int p0 = 0; p0 < NPIECE; p0 += RP) {
            uint32_t v[RP][16];
#pragma unroll
            for (int j = 0; j < RP; ++j)
              tmem_ld16(tmem + lane_base + (uint32_t)(b * BN) + (uint32_t)(col0 + 16 * (p0 + j)), v[j]);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < RP; ++j)
#pragma unroll
              for (int e = 0; e < 16; ++e) acc[16 * (p0 + j) + e] += __uint_as_float(v[j][e]);
          }
        }
        // the warp's TMEM loads are complete (wait::ld above); one lane
        // releases the buffer for the whole warp
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce[b]);
        ++cc;
      }
      if (!ok || !active) continue;
      // the tile's rows go out from registers while the MMAs of the next
      // tile fill the (now drained) TMEM buffers
      const int64_t row = tm * BM + q * 32 + lane;
      if (row >= M) continue;
#pragma unroll
      for (int pp = 0; pp < NPIECE; ++pp) {
        const int cl = col0 + 16 * pp;             // column within the tile
        const int f = cl / br;                     // pattern of the fold
        const int64_t pc = pc0 + f;
        const int64_t col = tn_ * br + (cl - f * br);
        if (pc >= PC) continue;
        float* crow = C + (pc * M + row) * N2;
        float w[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) w[e] = FMT == 2 ? (acc[16 * pp + e] * ua) * ub : acc[16 * pp + e];
        if (amax_out) {
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (col + e < N2) tmax = fmaxf(tmax, fabsf(acc[16 * pp + e]));
        }
        if (col + 16 <= N2) {
          float4* dst = (float4*)(crow + col);
#pragma unroll
          for (int e = 0; e < 4; ++e) dst[e] = make_float4(w[4 * e], w[4 * e + 1], w[4 * e + 2], w[4 * e + 3]);
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (col + e < N2) crow[col + e] = w[e];
        }
      }
    }
    if (amax_out && active) {
      // warp maximum, then the CTA maximum in shared memory (one global
      // atomic per CTA after the final barrier); unscaling by powers of two is
      // monotonic, so the maximum is scaled once
      if (FMT == 2) tmax = (tmax * ua) * ub;
      const unsigned int m = __reduce_max_sync(0xffffffffu, __float_as_uint(tmax));
      if (lane == 0) atomicMax(s_amax, m);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicOr(status, 1u);
  if (amax_out && threadIdx.x == 0 && *s_amax) atomicMax(amax_out, *s_amax);
  if (warp == 9) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Lay::TMEM_COLS));
  }
}

// ------------------------------------------------ CTA-pair variant (cta_group::2)
//
// Two CTAs of a cluster compute one 256 x 256 tile with 2-SM MMAs: CTA r holds
// rows [128 r, 128 r + 128) of the A tile and half of the B tile (its 128
// columns) in its own shared memory, and keeps its 128 rows x 256 columns of
// the accumulator in its own TMEM.  Each SM so reads half the B tile per MMA,
// which cuts shared-memory traffic by about a third against the one-CTA
// 128 x 256 tile and frees shared memory for more pipeline stages.
//   - The leader (rank 0) issues every MMA and commits them to the barriers of
//     both CTAs at once (multicast): a stage is free, a chunk is accumulated.
//   - Both CTAs' TMA loads complete on the leader's stage barrier, which the
//     leader arms with the bytes of both halves.
//   - The drain warps of both CTAs release a TMEM chunk buffer by arriving on
//     the leader's barrier (the peer's arrive is remote).
//   - TMEM is allocated and freed by one warp of each CTA together.
// Waits are bounded as in the one-CTA kernel; both CTAs meet at a cluster
// barrier before freeing TMEM and exiting, so neither leaves while the other
// may still touch its shared memory.

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// shared::cluster address of the same shared-memory location in CTA `rank`
__device__ __forceinline__ uint32_t mapa_rank(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Arrive on an mbarrier of another CTA of the cluster.  The arrive only has to
// order this warp's finished TMEM reads (tcgen05.wait::ld, then
// tcgen05.fence::before_thread_sync) before the leader's next MMA into the same
// columns, so it keeps the default CTA-scope release: a cluster-scope release
// would first wait for the previous tile's global stores of C to become
// visible across the cluster, which stalled the drain warps on every chunk.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

__device__ __forceinline__ void tma_load_3d_pair(void* dst, const CUtensorMap* map, uint32_t mbar_cluster, int c0,
                                                 int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
      "%4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(mbar_cluster)
      : "memory");
}

__device__ __forceinline__ void mma2(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// arrive on barrier `bar` (a local offset) in both CTAs of the pair once the
// MMAs issued so far complete
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar) {
  const uint16_t mask = 3;
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(mask)
      : "memory");
}

template <int STAGES>
struct LayoutPair {
  static constexpr int KB = 64;                   // 64-byte k-blocks (64-byte swizzle)
  static constexpr int A_BYTES = BM * KB;         // this CTA's 128 rows
  static constexpr int B_BYTES = 128 * KB;        // this CTA's half of the 256-row B tile
  static constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int DATA = STAGES * STAGE;
  static constexpr int TOTAL = DATA + 1024 + 256;
  static_assert(TOTAL <= 232448, "shared memory per CTA");
  static_assert(2 * STAGES + 8 <= 32, "barrier area");
  static constexpr uint32_t TMEM_COLS = 512;     // two chunk buffers of 256 fp32 columns
};

// Instruction descriptor of a 256 x 256 pair MMA (kind::f16, fp32 accumulate)
template <int FMT>
__device__ __forceinline__ uint32_t idesc_pair() {
  const uint32_t f = FMT == 1 ? 1u : 0u;
  return (1u << 4) | (f << 7) | (f << 10) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);
}

template <int STAGES, int FMT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    k_gemm_tc_pair(const __grid_constant__ CUtensorMap tmAhi, const __grid_constant__ CUtensorMap tmAlo,
                   const __grid_constant__ CUtensorMap tmBhi, const __grid_constant__ CUtensorMap tmBlo,
                   float* __restrict__ C, int64_t M, int64_t N2, int64_t K2, int64_t tilesM, int64_t tilesN,
                   int64_t PC, int64_t PCg, int fold, const uint32_t* __restrict__ mapA,
                   const uint32_t* __restrict__ mapB, int mapA_mode, int mapB_mode, const unsigned int* scaleA,
                   const unsigned int* scaleB, unsigned int* amax_out, unsigned int* status) {
  static_assert(FMT == 1 || FMT == 2, "pair MMAs use kind::f16 operands");
  constexpr int BN = 256;
  using Lay = LayoutPair<STAGES>;
  constexpr int KB = Lay::KB;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + Lay::DATA);
  uint64_t* full = bars;                    // leader: stage loaded in both CTAs  [STAGES]
  uint64_t* empty = bars + STAGES;          // both: stage consumed               [STAGES]
  uint64_t* accf = bars + 2 * STAGES;       // both: chunk accumulated            [2]
  uint64_t* acce = bars + 2 * STAGES + 2;   // leader: chunk drained in both CTAs [2]
  uint64_t* mma_done = bars + 2 * STAGES + 4;
  volatile uint32_t* tmem_slot = (volatile uint32_t*)(bars + 2 * STAGES + 5);
  volatile int* abort_flag = (volatile int*)(bars + 2 * STAGES + 6);
  unsigned int* s_amax = (unsigned int*)(bars + 2 * STAGES + 7);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int64_t cluster = blockIdx.x >> 1, n_clusters = gridDim.x >> 1;
  const bool a_shared = mapA_mode == 1 && PC > 1;
  const int64_t n_tiles = tilesM * tilesN * PCg;
  const int br = BN / fold;                 // B rows per pattern box (2N when folded)
  const int half_boxes = fold >= 2 ? fold / 2 : 1;   // B boxes this CTA loads per stage
  const int box_rows = fold >= 2 ? br : 128;
  constexpr int BKE = KB / 2;               // K elements (16-bit) per k-block
  constexpr int CH = chunk_bytes(FMT) / KB, KK = KBlock<KB>::KK;
  const int nkb = (int)((K2 + BKE - 1) / BKE);
  const int nch = (nkb + CH - 1) / CH;
  auto coords = [&](int64_t t, int64_t& pc0, int64_t& tm, int64_t& tn_) {
    int64_t pg;
    tile_coords(t, tilesM, tilesN, PCg, a_shared, pg, tm, tn_);
    pc0 = pg * fold;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 16);              // one arrive per drain warp of each CTA
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    *s_amax = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 9) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32((const void*)tmem_slot)),
                 "r"(Lay::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  cluster_sync_all();                       // both CTAs' barriers exist before any remote use
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;

  if (warp == 8) {
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int64_t t = cluster; t < n_tiles && ok; t += n_clusters) {
        int64_t pc0, tm, tn_;
        coords(t, pc0, tm, tn_);
        const int64_t pa = mapA_mode == 0 ? pc0 : (mapA_mode == 1 ? 0 : (int64_t)mapA[pc0]);
        const int row0 = (int)(tm * 2 * BM + rank * BM);
        for (int kb = 0; kb < nkb; ++kb) {
          const int s = (int)(it % STAGES);
          const uint32_t r = it / STAGES;
          if (!mbar_wait(&empty[s], (r & 1) ^ 1, abort_flag)) { ok = false; break; }
          const uint32_t fb = mapa_rank(smem_u32(&full[s]), 0);
          if (leader) mbar_expect_tx(&full[s], (uint32_t)(2 * Lay::STAGE));   // both CTAs' halves
          uint8_t* st = smem + s * Lay::STAGE;
          tma_load_3d_pair(st, &tmAhi, fb, kb * BKE, row0, (int)pa);
          tma_load_3d_pair(st + Lay::A_BYTES, &tmAlo, fb, kb * BKE, row0, (int)pa);
          for (int h = 0; h < half_boxes; ++h) {
            int64_t pcf = pc0;
            int nrow = (int)(tn_ * BN + rank * 128);
            if (fold >= 2) {
              const int f = (int)rank * half_boxes + h;
              pcf = pc0 + f < PC ? pc0 + f : PC - 1;
              nrow = 0;
            }
            const int64_t pb = mapB_mode == 0 ? pcf : (mapB_mode == 1 ? 0 : (int64_t)mapB[pcf]);
            uint8_t* sb = st + 2 * Lay::A_BYTES + h * box_rows * KB;
            tma_load_3d_pair(sb, &tmBhi, fb, kb * BKE, nrow, (int)pb);
            tma_load_3d_pair(sb + Lay::B_BYTES, &tmBlo, fb, kb * BKE, nrow, (int)pb);
          }
          ++it;
        }
      }
      if (!ok) {
        // The copies of both CTAs complete on the leader's stage barriers: the
        // leader waits out its last STAGES k-blocks there.  The peer cannot
        // observe its own copies (their barrier is the leader's), and the two
        // producers may stop one k-block apart, so both also hold for a
        // bounded time (about a millisecond) before the final cluster barrier.
        if (leader)
          for (uint32_t j = it > (uint32_t)STAGES ? it - STAGES : 0; j < it; ++j)
            mbar_drain(&full[j % STAGES], (j / STAGES) & 1);
        const long long t0 = clock64();
        while (clock64() - t0 < (1LL << 21)) {
        }
      }
    }
  } else if (warp == 9) {
    if (lane == 0 && leader) {
      const uint32_t idesc = idesc_pair<FMT>();
      uint32_t it = 0, cc = 0;
      bool ok = true;
      for (int64_t t = cluster; t < n_tiles && ok; t += n_clusters) {
        for (int kb = 0; kb < nkb; ++kb) {
          const int s = (int)(it % STAGES);
          const uint32_t r = it / STAGES;
          const int b = (int)(cc & 1);
          const uint32_t u = cc >> 1;
          const bool first = kb % CH == 0, last = kb % CH == CH - 1 || kb == nkb - 1;
          if (first && !mbar_wait(&acce[b], (u & 1) ^ 1, abort_flag)) { ok = false; break; }
          if (!mbar_wait(&full[s], r & 1, abort_flag)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t d = tmem + (uint32_t)(b * BN);
          const uint32_t st = smem_u32(smem + s * Lay::STAGE);
          const uint32_t a_hi = st, a_lo = st + Lay::A_BYTES;
          const uint32_t b_hi = st + 2 * Lay::A_BYTES, b_lo = b_hi + Lay::B_BYTES;
#pragma unroll
          for (int kk = 0; kk < KK; ++kk) {
            const uint32_t o = kk * 32;
            mma2(d, sdesc<KB>(a_hi + o), sdesc<KB>(b_lo + o), idesc, (first && kk == 0) ? 0u : 1u);
            mma2(d, sdesc<KB>(a_lo + o), sdesc<KB>(b_hi + o), idesc, 1u);
          }
#pragma unroll
          for (int kk = 0; kk < KK; ++kk) {
            const uint32_t o = kk * 32;
            mma2(d, sdesc<KB>(a_hi + o), sdesc<KB>(b_hi + o), idesc, 1u);
          }
          mma_commit_pair(&empty[s]);
          if (last) {
            mma_commit_pair(&accf[b]);
            ++cc;
          }
          ++it;
        }
      }
      // every issued MMA (they write both CTAs' TMEM) completes before either
      // CTA frees TMEM; a commit with nothing pending arrives at once
      mma_commit_pair(mma_done);
    }
  } else {
    // drain warps 0-7 of both CTAs: this CTA's 128 rows, 128 columns per warp
    constexpr int NCOL = BN / 2;
    constexpr int NPIECE = NCOL / 16;
    constexpr int RP = 2;
    const int q = warp & 3, half = warp >> 2;
    const int col0 = half * NCOL;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const float ua = FMT == 2 ? pow2f(-fp16_scale_exp(*scaleA)) : 1.0f;
    const float ub = FMT == 2 ? pow2f(-fp16_scale_exp(*scaleB)) : 1.0f;
    // the leader's release barriers: acce[b] sits 8 bytes past acce[0] there
    // too (an offset, not an indexed local array, which would live in local
    // memory)
    const uint32_t acce_leader = mapa_rank(smem_u32(&acce[0]), 0);
    float tmax = 0.0f;
    uint32_t cc = 0;
    bool ok = true;
    for (int64_t t = cluster; t < n_tiles && ok; t += n_clusters) {
      int64_t pc0, tm, tn_;
      coords(t, pc0, tm, tn_);
      float acc[NCOL];
#pragma unroll
      for (int e = 0; e < NCOL; ++e) acc[e] = 0.0f;
      for (int c = 0; c < nch; ++c) {
        const int b = (int)(cc & 1);
        const uint32_t u = cc >> 1;
        ok = mbar_wait(&accf[b], u & 1, abort_flag);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
        for (int p0 = 0; p0 < NPIECE; p0 += RP) {
          uint32_t v[RP][16];
#pragma unroll
          for (int j = 0; j < RP; ++j)
            tmem_ld16(tmem + lane_base + (uint32_t)(b * BN) + (uint32_t)(col0 + 16 * (p0 + j)), v[j]);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < RP; ++j)
#pragma unroll
            for (int e = 0; e < 16; ++e) acc[16 * (p0 + j) + e] += __uint_as_float(v[j][e]);
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(acce_leader + 8u * (uint32_t)b);
        ++cc;
      }
      if (!ok) continue;
      const int64_t row = tm * 2 * BM + (int64_t)rank * BM + q * 32 + lane;
      if (row >= M) continue;
#pragma unroll
      for (int pp = 0; pp < NPIECE; ++pp) {
        const int cl = col0 + 16 * pp;
        const int f = cl / br;
        const int64_t pc = pc0 + f;
        const int64_t col = tn_ * br + (cl - f * br);
        if (pc >= PC) continue;
        float* crow = C + (pc * M + row) * N2;
        float w[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) w[e] = FMT == 2 ? (acc[16 * pp + e] * ua) * ub : acc[16 * pp + e];
        if (amax_out) {
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (col + e < N2) tmax = fmaxf(tmax, fabsf(acc[16 * pp + e]));
        }
        if (col + 16 <= N2) {
          float4* dst = (float4*)(crow + col);
#pragma unroll
          for (int e = 0; e < 4; ++e) dst[e] = make_float4(w[4 * e], w[4 * e + 1], w[4 * e + 2], w[4 * e + 3]);
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (col + e < N2) crow[col + e] = w[e];
        }
      }
    }
    if (amax_out) {
      if (FMT == 2) tmax = (tmax * ua) * ub;
      const unsigned int m = __reduce_max_sync(0xffffffffu, __float_as_uint(tmax));
      if (lane == 0) atomicMax(s_amax, m);
    }
  }
  // both CTAs: wait (bounded) until the leader's MMAs are complete, then meet
  if (threadIdx.x == 0) mbar_drain(mma_done, 0);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  cluster_sync_all();
  if (*abort_flag && threadIdx.x == 0) atomicOr(status, 1u);
  if (amax_out && threadIdx.x == 0 && *s_amax) atomicMax(amax_out, *s_amax);
  if (warp == 9) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Lay::TMEM_COLS));
  }
}

// ------------------------------------------------------------------ host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

static bool encode3d(CUtensorMap* m, const void* base, uint64_t d0, uint64_t d1, uint64_t d2, uint32_t b0,
                     uint32_t b1, int fmt, int kb) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[3] = {d0, d1, d2};
  const uint64_t es_bytes = fmt ? 2 : 4;
  const CUtensorMapDataType dt = fmt == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : fmt == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                            : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  cuuint64_t strides[2] = {d0 * es_bytes, d0 * d1 * es_bytes};
  cuuint32_t box[3] = {b0, b1, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(m, dt, 3, const_cast<void*>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE,
                   kb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int BN, int STAGES, int FMT>
static cudaError_t set_attr() {
  constexpr int KB = kb_bytes(BN, FMT);
  using Lay = Layout<BN, STAGES, KB>;
  return cudaFuncSetAttribute(k_gemm_tc<BN, STAGES, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::TOTAL);
}

static int sm_count() {
  static int n[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (!n[dev] && cudaDeviceGetAttribute(&n[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n[dev] = 152;
  return n[dev] > 0 ? n[dev] : 152;
}

// fold = patterns per tile side by side along N (1: none); see the kernel
template <int BN, int STAGES, int FMT>
static cudaError_t run(const GemmParams& p, int fold, unsigned int* status, cudaStream_t s) {
  constexpr int KB = kb_bytes(BN, FMT);
  using Lay = Layout<BN, STAGES, KB>;
  const int64_t K2 = 2 * p.K, N2 = 2 * p.N;
  const int br = BN / fold;
  if (fold > 1 && (br != N2 || br < 16 || p.mapA_mode != 1)) return cudaErrorInvalidValue;
  const uint32_t BKE = KB / (FMT ? 2 : 4);
  const int64_t es = FMT ? 2 : 4;
  // A: hi plane then lo plane, each [PA][M][2K]; B: hi plane then lo plane, each [PB][2N][2K]
  const char* ahi = (const char*)p.A;
  const char* alo = ahi + p.PA * p.M * K2 * es;
  const char* bhi = (const char*)p.B;
  const char* blo = bhi + p.PB * N2 * K2 * es;
  CUtensorMap tah, tal, tbh, tbl;
  if (!encode3d(&tah, ahi, (uint64_t)K2, (uint64_t)p.M, (uint64_t)p.PA, BKE, BM, FMT, KB)) return cudaErrorInvalidValue;
  if (!encode3d(&tal, alo, (uint64_t)K2, (uint64_t)p.M, (uint64_t)p.PA, BKE, BM, FMT, KB)) return cudaErrorInvalidValue;
  if (!encode3d(&tbh, bhi, (uint64_t)K2, (uint64_t)N2, (uint64_t)p.PB, BKE, br, FMT, KB)) return cudaErrorInvalidValue;
  if (!encode3d(&tbl, blo, (uint64_t)K2, (uint64_t)N2, (uint64_t)p.PB, BKE, br, FMT, KB)) return cudaErrorInvalidValue;
  const int64_t tilesM = (p.M + BM - 1) / BM, tilesN = fold > 1 ? 1 : (N2 + BN - 1) / BN;
  const int64_t PCg = (p.PC + fold - 1) / fold;
  const int64_t n_tiles = tilesM * tilesN * PCg;
  if (n_tiles <= 0) return cudaSuccess;
  // persistent: at most one CTA per SM (the pipeline's shared memory allows one)
  const int64_t grid = std::min<int64_t>(n_tiles, sm_count());
  k_gemm_tc<BN, STAGES, FMT><<<(unsigned)grid, kThreads, Lay::TOTAL, s>>>(
      tah, tal, tbh, tbl, (float*)p.C, p.M, N2, K2, tilesM, tilesN, p.PC, PCg, fold, p.mapA, p.mapB, p.mapA_mode,
      p.mapB_mode, p.scaleA, p.scaleB, p.amax, status);
  return cudaGetLastError();
}

constexpr int kPairStages = 6;

template <int FMT>
static cudaError_t set_attr_pair() {
  return cudaFuncSetAttribute(k_gemm_tc_pair<kPairStages, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              LayoutPair<kPairStages>::TOTAL);
}

// The CTA-pair kernel: 256 x 256 tiles on clusters of two CTAs.
template <int FMT>
static cudaError_t run_pair(const GemmParams& p, int fold, unsigned int* status, cudaStream_t s) {
  using Lay = LayoutPair<kPairStages>;
  constexpr int BN = 256, KB = Lay::KB;
  const int64_t K2 = 2 * p.K, N2 = 2 * p.N;
  const int br = BN / fold;
  if (fold > 1 && (br != N2 || br < 16 || p.mapA_mode != 1 || fold % 2)) return cudaErrorInvalidValue;
  const uint32_t BKE = KB / 2;
  const int64_t es = 2;
  const char* ahi = (const char*)p.A;
  const char* alo = ahi + p.PA * p.M * K2 * es;
  const char* bhi = (const char*)p.B;
  const char* blo = bhi + p.PB * N2 * K2 * es;
  const uint32_t box_rows = fold >= 2 ? (uint32_t)br : 128u;
  CUtensorMap tah, tal, tbh, tbl;
  if (!encode3d(&tah, ahi, (uint64_t)K2, (uint64_t)p.M, (uint64_t)p.PA, BKE, BM, FMT, KB)) return cudaErrorInvalidValue;
  if (!encode3d(&tal, alo, (uint64_t)K2, (uint64_t)p.M, (uint64_t)p.PA, BKE, BM, FMT, KB)) return cudaErrorInvalidValue;
  if (!encode3d(&tbh, bhi, (uint64_t)K2, (uint64_t)N2, (uint64_t)p.PB, BKE, box_rows, FMT, KB))
    return cudaErrorInvalidValue;
  if (!encode3d(&tbl, blo, (uint64_t)K2, (uint64_t)N2, (uint64_t)p.PB, BKE, box_rows, FMT, KB))
    return cudaErrorInvalidValue;
  const int64_t tilesM = (p.M + 2 * BM - 1) / (2 * BM), tilesN = fold > 1 ? 1 : (N2 + BN - 1) / BN;
  const int64_t PCg = (p.PC + fold - 1) / fold;
  const int64_t n_tiles = tilesM * tilesN * PCg;
  if (n_tiles <= 0) return cudaSuccess;
  const int64_t clusters = std::min<int64_t>(n_tiles, sm_count() / 2);
  k_gemm_tc_pair<kPairStages, FMT><<<(unsigned)(2 * clusters), kThreads, Lay::TOTAL, s>>>(
      tah, tal, tbh, tbl, (float*)p.C, p.M, N2, K2, tilesM, tilesN, p.PC, PCg, fold, p.mapA, p.mapB, p.mapA_mode,
      p.mapB_mode, p.scaleA, p.scaleB, p.amax, status);
  return cudaGetLastError();
}

}  // namespace tc

// Tile width: the smallest of 16..cap (cap = p.tile_cap, a power of two in
// 16..256; 256 by default) that covers 2N, or, when all patterns share A and
// 2N >= 16, up to cap columns of consecutive patterns folded side by side
// (fold = BN / 2N, as many as the pattern count rounded up to a power of two
// allows).  256-wide 16-bit tiles with at least 256 rows run on CTA pairs
// unless p.pair < 0.
GemmTile gemm_tc_tile(const GemmParams& p) {
  int cap = 16;
  while (cap < 256 && cap < p.tile_cap) cap *= 2;
  const int64_t N2 = 2 * p.N;
  int64_t w = N2;
  int fold = 1;
  if (p.mapA_mode == 1 && p.PC > 1 && N2 >= 16 && N2 < cap) {
    while (w < cap && fold < p.PC) {
      w *= 2;
      fold *= 2;
    }
  }
  GemmTile t;
  t.bn = 16;
  while (t.bn < 256 && t.bn < std::min<int64_t>(w, cap)) t.bn *= 2;
  t.fold = fold;
  t.paired = p.h16 != 0 && t.bn == 256 && p.M >= 2 * tc::BM && p.pair >= 0;
  return t;
}

namespace tc {

template <int FMT>
static cudaError_t dispatch(const GemmParams& p, unsigned int* status, cudaStream_t s) {
  const GemmTile t = gemm_tc_tile(p);
  const int fold = t.fold;
  if (t.bn == 16) return run<16, kb_stages(16, kb_bytes(16, FMT)), FMT>(p, fold, status, s);
  if (t.bn == 32) return run<32, kb_stages(32, kb_bytes(32, FMT)), FMT>(p, fold, status, s);
  if (t.bn == 64) return run<64, kb_stages(64, kb_bytes(64, FMT)), FMT>(p, fold, status, s);
  if (t.bn == 128) return run<128, kb_stages(128, kb_bytes(128, FMT)), FMT>(p, fold, status, s);
  if (t.paired) return run_pair<FMT == 0 ? 1 : FMT>(p, fold, status, s);
  return run<256, kb_stages(256, kb_bytes(256, FMT)), FMT>(p, fold, status, s);
}

template <int FMT>
static cudaError_t set_attrs() {
  if (FMT != 0) {
    const cudaError_t e = set_attr_pair<FMT == 0 ? 1 : FMT>();
    if (e != cudaSuccess) return e;
  }
  const cudaError_t r[5] = {set_attr<16, kb_stages(16, kb_bytes(16, FMT)), FMT>(),
                            set_attr<32, kb_stages(32, kb_bytes(32, FMT)), FMT>(),
                            set_attr<64, kb_stages(64, kb_bytes(64, FMT)), FMT>(),
                            set_attr<128, kb_stages(128, kb_bytes(128, FMT)), FMT>(),
                            set_attr<256, kb_stages(256, kb_bytes(256, FMT)), FMT>()};
  for (cudaError_t x : r)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}

}  // namespace tc

cudaError_t prepare_gemm_tc() {
  // the opt-in shared-memory size and the SM count, set once per device before
  // any launch (and so before any stream capture)
  tc::sm_count();
  cudaError_t e = tc::set_attrs<0>();
  const cudaError_t e1 = tc::set_attrs<1>(), e2 = tc::set_attrs<2>();
  if (e == cudaSuccess) e = e1;
  if (e == cudaSuccess) e = e2;
  return e;
}

cudaError_t launch_gemm_tc(const GemmParams& p, unsigned int* status, cudaStream_t s) {
  // row pitch of A (2K elements) must be a multiple of 16 bytes
  if (p.K < (p.h16 ? 4 : 2)) return cudaErrorInvalidValue;
  if (p.h16 == 2) return tc::dispatch<2>(p, status, s);
  if (p.h16 == 1) return tc::dispatch<1>(p, status, s);
  return tc::dispatch<0>(p, status, s);
}

}  // namespace tn
