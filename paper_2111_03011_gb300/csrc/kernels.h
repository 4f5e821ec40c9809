// Device kernels of the contraction path and their launch parameters.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace tn {

// Operand scaling of the FP16x3 engine.  An ABSMAX step writes m = max over a
// GEMM operand of |re| and |im| (as fp32 bits, by atomicMax) into a scale slot.
// The split kernels multiply the operand by 2^k with k = 14 - floor(log2 m)
// (so that |x| 2^k < 2^15 < 65504, the fp16 maximum, while the largest entries
// and their split remainders keep full fp16 precision); the GEMM epilogue
// multiplies by 2^-kA 2^-kB.  Powers of two: every scaling is exact.
__host__ __device__ __forceinline__ int fp16_scale_exp(unsigned int m_bits) {
  if (m_bits == 0) return 14;                       // all-zero operand
  int e = (int)((m_bits >> 23) & 0xffu) - 127;      // floor(log2 m) for normal m
  if (e < -100) e = -100;
  return 14 - e;                                    // in [14 - 127, 114]
}
// 2^k as an fp32, for -126 <= k <= 127 (built from its exponent bits)
__host__ __device__ __forceinline__ float pow2f(int k) {
  union { unsigned int u; float f; } x;
  x.u = (unsigned int)(127 + k) << 23;
  return x.f;
}

struct AbsmaxParams {
  const float2* in;
  int64_t n;             // complex elements
  unsigned int* out;     // scale slot (fp32 bits of the running maximum; zeroed per pass)
};

// C[p][m + (n << (rA-nk))] = sum_k A[mapA(p)][insert_K(m) + k-offset] * B[mapB(p)][boffK[k] + boffN[n]]
struct SmallParams {
  const float2* A; const float2* B; float2* C;
  int64_t a_pstride, b_pstride, c_pstride;
  int64_t M;            // rows per pattern = 2^(rA - nk)
  int64_t PC;
  int rA, nk, nn;
  int kpos[4];
  uint32_t boffK[16], boffN[16];
  const uint32_t* mapA; const uint32_t* mapB;
  int mapA_mode, mapB_mode;  // 0 identity, 1 zero, 2 table
  unsigned int* amax;        // non-null: atomicMax of the output's max |re|, |im| (fp32 bits)
};

// out[p][bo + out_off[j]] = in[p][bi + in_off[slot[j]]], (bi, bo) from the rest bits
struct PermParams {
  const float2* in; float2* out;
  int64_t pstride, P;
  int t;                 // tile bits
  int n_rest;
  uint8_t rest_in[64], rest_out[64];
  const uint32_t* tab;   // in_off[2^t], out_off[2^t], slot[2^t]
  int split;             // 1: write tf32 hi plane then lo plane (fp32 pairs); 2: bf16 planes;
                         // 3: fp16 planes of the value times 2^k (k from *scale);
                         // 4, 5, 6: the tensor-core B operand (real embedding of the permuted
                         // [N][K] tensor) in tf32, bf16 or scaled fp16 hi/lo planes
  const unsigned int* scale;   // SPLIT 3: the operand's scale slot
  int vec4 = 0;          // 1: output bits 0 and 1 are tile bits 0 and 1 (four outputs per store)
  int embed_nk = 0;      // split 4-6: log2 K (the output's low bits are the K legs)
};

struct BPrepParams {
  const float2* B; void* out;
  int64_t b_pstride, PB;
  int nk, nn;
  const uint32_t* bk; const uint32_t* bn;
  int h16;               // tensor-core B: 0 tf32 planes, 1 bf16 planes, 2 scaled fp16 planes
  const unsigned int* scale;   // h16 == 2: the operand's scale slot
};

// C[p][m][n] = sum_k A[mapA(p)][m][k] B[mapB(p)][k][n]
struct GemmParams {
  const float2* A; const void* B; float2* C;
  int64_t M, N, K;      // complex dimensions (powers of two)
  int64_t PA, PB, PC;
  const uint32_t* mapA; const uint32_t* mapB;
  int mapA_mode, mapB_mode;
  int h16;               // tensor-core engine: 0 tf32, 1 bf16, 2 scaled fp16 hi/lo operand planes
  const unsigned int* scaleA; const unsigned int* scaleB;   // h16 == 2: the operands' scale slots
  unsigned int* amax;    // non-null: atomicMax of the output's max |re|, |im| (fp32 bits)
  int pair = 0;          // 0: CTA-pair 256 x 256 tiles where they apply (16-bit, M >= 256); -1: one-CTA tiles
  int tile_cap = 256;    // widest tile the dispatch may pick, real columns (16..256)
};

// Tile a tensor-core GEMM launch runs with: BN real columns per tile, fold
// patterns side by side in one tile, on CTA pairs or not.
struct GemmTile {
  int bn = 256, fold = 1;
  bool paired = false;
};
GemmTile gemm_tc_tile(const GemmParams& p);

struct AccumParams {
  const float2* F; double2* H;
  int64_t f_pstride;
  int64_t L; int h;
  const uint32_t* pidx;
  int open_pos[32];
};

cudaError_t launch_small(const SmallParams& p, cudaStream_t s);
cudaError_t launch_absmax(const AbsmaxParams& p, cudaStream_t s);
cudaError_t launch_permute(const PermParams& p, cudaStream_t s);
cudaError_t launch_bprep_c(const BPrepParams& p, cudaStream_t s);
cudaError_t launch_bprep_tc(const BPrepParams& p, cudaStream_t s, bool beside_gemm = false);
cudaError_t launch_gemm_simt(const GemmParams& p, cudaStream_t s);
cudaError_t launch_accum(const AccumParams& p, cudaStream_t s);

// Tensor-core GEMM (gemm_tc.cu).  A = hi then lo fp32 planes [PA][M][2K];
// B = real-embedded hi then lo planes [PB][2N][2K].
// `status` receives a nonzero code if a bounded wait gave up.
cudaError_t launch_gemm_tc(const GemmParams& p, unsigned int* status, cudaStream_t s);
cudaError_t prepare_gemm_tc();   // kernel attributes; call before launching or capturing
cudaError_t prepare_permute();   // the permute's opt-in shared-memory size; likewise

// amplitude lookup: out[i] = H[g][mu] (c128 or c64); status <- min missing
// index, or with seg_end (cumulative ends of n_seg merged requests, device)
// status[j] <- min missing index within request j
cudaError_t launch_amplitudes(const double2* H, int h, const uint64_t* keys, const uint32_t* groups, int64_t n_keys,
                              uint64_t tail_mask, const int* open_q, const uint64_t* bits, int64_t n, void* out,
                              int dtype, unsigned long long* status, cudaStream_t s, const int64_t* seg_end = nullptr,
                              int n_seg = 1);

// per-group squared norms Z[g] (chunked warp order) and the total N
cudaError_t launch_group_norms(const double2* H, int64_t L, int h, double* Z, double* N, cudaStream_t s);

// sums[0] = sum |a_i|^2, sums[1] = sum log |a_i|^2 over n complex128 amplitudes
// (FP64; `part` holds xeb_partials(n) doubles of scratch)
cudaError_t launch_xeb_sums(const double2* amp, int64_t n, double* part, double* sums, cudaStream_t s);
int64_t xeb_partials(int64_t n);

struct SampleParams {
  const double2* H; int64_t L; int h;
  const uint64_t* tails; uint64_t open_mask; const int* open_q;
  int n_qubits;
  int64_t n;
  double mix;                 // probability of a uniform draw
  uint64_t seed;
  uint64_t* out;
  int method;                 // 0 exact inverse CDF, 1 Metropolis chain, 2 frugal rejection
  int64_t param;              // chain length (1) or the bound M (2)
};
cudaError_t launch_sample(const SampleParams& p, cudaStream_t s);

}  // namespace tn
