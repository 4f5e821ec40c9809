// Streaming kernels of the contraction path (HBM-bound steps), the plain
// FP32 CUDA-core complex GEMM, slice accumulation, amplitude lookup, norms and
// the group sampler.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdio>

#include "kernels.h"

namespace tn {

static constexpr int kSMs = 152;

__device__ __forceinline__ int64_t map_p(int mode, const uint32_t* tab, int64_t p) {
  return mode == 0 ? p : (mode == 1 ? 0 : (int64_t)__ldg(tab + p));
}

__device__ __forceinline__ float2 cmul_add(float2 acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
  return acc;
}

// ------------------------------------------------------------------ K8 / K3
// Small-operand contraction (a gate-like tensor of <= 16x16 applied to a big
// one).  Each thread owns one row m of the big operand: it gathers the 2^NK
// elements addressed by the contracted legs, multiplies by the small operand
// held in shared memory, and writes 2^NN outputs.  Consecutive threads touch
// consecutive addresses, so loads and stores coalesce whatever the leg layout.
template <int NK, int NN>
__global__ void __launch_bounds__(256) k_small(SmallParams p) {
  constexpr int KK = 1 << NK, NNN = 1 << NN;
  __shared__ float2 Bs[KK][NNN];
  int64_t offK[KK];
#pragma unroll
  for (int k = 0; k < KK; ++k) {
    int64_t o = 0;
#pragma unroll
    for (int j = 0; j < NK; ++j)
      if ((k >> j) & 1) o |= 1LL << p.kpos[j];
    offK[k] = o;
  }
  const int64_t rowsC = p.M;  // C stride of the n index
  __shared__ unsigned int s_amax;
  if (threadIdx.x == 0) s_amax = 0u;
  float tmax = 0.0f;
  for (int64_t pc = blockIdx.y; pc < p.PC; pc += gridDim.y) {
    const int64_t pa = map_p(p.mapA_mode, p.mapA, pc);
    const int64_t pb = map_p(p.mapB_mode, p.mapB, pc);
    __syncthreads();
    for (int i = threadIdx.x; i < KK * NNN; i += blockDim.x) {
      const int k = i / NNN, n = i % NNN;
      Bs[k][n] = p.B[pb * p.b_pstride + p.boffK[k] + p.boffN[n]];
    }
    __syncthreads();
    const float2* __restrict__ Ap = p.A + pa * p.a_pstride;
    float2* __restrict__ Cp = p.C + pc * p.c_pstride;
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < p.M; m += (int64_t)gridDim.x * blockDim.x) {
      int64_t x = m;
#pragma unroll
      for (int j = 0; j < NK; ++j) {
        const int pos = p.kpos[j];
        x = ((x >> pos) << (pos + 1)) | (x & ((1LL << pos) - 1));
      }
      float2 a[KK];
#pragma unroll
      for (int k = 0; k < KK; ++k) a[k] = __ldg(Ap + x + offK[k]);
#pragma unroll
      for (int n = 0; n < NNN; ++n) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < KK; ++k) acc = cmul_add(acc, a[k], Bs[k][n]);
        Cp[m + (int64_t)n * rowsC] = acc;
        tmax = fmaxf(tmax, fmaxf(fabsf(acc.x), fabsf(acc.y)));
      }
    }
  }
  if (p.amax) {
    // block maximum of the output (FP16x3 scale of the next GEMM operand)
    unsigned int b = __reduce_max_sync(0xffffffffu, __float_as_uint(tmax));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicMax(&s_amax, b);
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(p.amax, s_amax);
  }
}

template <int NK, int NN>
static cudaError_t launch_small_t(const SmallParams& p, cudaStream_t s) {
  const int threads = 256;
  int64_t bx = (p.M + threads - 1) / threads;
  const int64_t cap = (int64_t)kSMs * 8;
  int64_t by = p.PC < 65535 ? p.PC : 65535;
  if (bx * by > cap * 4) bx = std::max<int64_t>(1, (cap * 4) / by);
  if (bx < 1) bx = 1;
  k_small<NK, NN><<<dim3((unsigned)bx, (unsigned)by), threads, 0, s>>>(p);
  return cudaGetLastError();
}

typedef cudaError_t (*small_fn)(const SmallParams&, cudaStream_t);
#define SMALL_ROW(NK) {launch_small_t<NK, 0>, launch_small_t<NK, 1>, launch_small_t<NK, 2>, launch_small_t<NK, 3>, launch_small_t<NK, 4>}
static const small_fn small_table[5][5] = {SMALL_ROW(0), SMALL_ROW(1), SMALL_ROW(2), SMALL_ROW(3), SMALL_ROW(4)};

cudaError_t launch_small(const SmallParams& p, cudaStream_t s) {
  if (p.nk < 0 || p.nk > 4 || p.nn < 0 || p.nn > 4) return cudaErrorInvalidValue;
  return small_table[p.nk][p.nn](p, s);
}

// ---------------------------------------------------------------------- K1
// Bit-permutation transpose.  A tile covers the input's low bits and the
// preimages of the output's low bits (grown to 10 bits with further input
// bits); it is read with the input's contiguous order and written with the
// output's, through shared memory.  The tile is padded by one element per 32 so
// that the strided reads of the write phase fall into different banks.  The
// tile's base addresses (the remaining "rest" bits of the tile index scattered
// to their positions) come from one 256-entry table per byte of the rest bits
// and direction (only as many as n_rest needs, to keep shared memory small and
// more blocks, hence more loads, in flight per SM).
// SPLIT 1: the output is written as two fp32 planes, tf32-rounded hi and the
// remainder lo; SPLIT 2: two bf16 planes, bf16 hi and the bf16-rounded
// remainder; SPLIT 3: two fp16 planes of the value times the operand's power-
// of-two scale (fp16_scale_exp of its ABSMAX slot) -- the operand formats of
// the three tensor-core GEMM engines.
__device__ __forceinline__ int pad32(int i) { return i + (i >> 5); }

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Asynchronous 8-byte global -> shared copies (cp.async): the loads of the
// next tiles land in shared memory without holding registers.
__device__ __forceinline__ void cp_async8(float2* dst, const float2* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Tile buffers of the permute: while one tile is written out, the next
// kPermBufs - 1 are in flight.
constexpr int kPermBufs = 3;

__host__ __device__ inline int perm_levels(int n_rest) { return n_rest > 0 ? (n_rest + 7) >> 3 : 1; }
// float2 per buffer, even so that the index tables after the buffers start on 16 bytes
__host__ __device__ inline int perm_tile_stride(int nt) { return (nt + (nt >> 5) + 3) & ~1; }

// Four consecutive outputs of one plane as one 16-byte store (16-bit formats)
// or two (fp32 pairs); the destination index is a multiple of 4.
__device__ __forceinline__ void store4(float2* dst, float2 a, float2 b, float2 c, float2 d) {
  float4* q = (float4*)dst;
  q[0] = make_float4(a.x, a.y, b.x, b.y);
  q[1] = make_float4(c.x, c.y, d.x, d.y);
}
template <typename H2>
__device__ __forceinline__ void store4(H2* dst, H2 a, H2 b, H2 c, H2 d) {
  *(uint4*)dst = make_uint4(*(const uint32_t*)&a, *(const uint32_t*)&b, *(const uint32_t*)&c, *(const uint32_t*)&d);
}

// Split of two reals into the hi and lo parts of a tensor-core operand format
// (FMT 0: tf32-rounded fp32 hi + fp32 remainder; 1: bf16 hi + bf16 remainder;
// 2: fp16 of the value times the scale sc).
template <int FMT>
struct Pair;
template <>
struct Pair<0> {
  using T = float2;
  static __device__ __forceinline__ void split(float a, float b, float, T& h, T& l) {
    h = make_float2(tf32_rn(a), tf32_rn(b));
    l = make_float2(a - h.x, b - h.y);
  }
};
template <>
struct Pair<1> {
  using T = __nv_bfloat162;
  static __device__ __forceinline__ void split(float a, float b, float, T& h, T& l) {
    h = __floats2bfloat162_rn(a, b);
    const float2 f = __bfloat1622float2(h);
    l = __floats2bfloat162_rn(a - f.x, b - f.y);
  }
};
template <>
struct Pair<2> {
  using T = __half2;
  static __device__ __forceinline__ void split(float a, float b, float sc, T& h, T& l) {
    a *= sc;
    b *= sc;
    h = __floats2half2_rn(a, b);
    const float2 f = __half22float2(h);
    l = __floats2half2_rn(a - f.x, b - f.y);
  }
};

template <int SPLIT>
__global__ void __launch_bounds__(256) k_permute(PermParams p) {
  extern __shared__ float2 tile[];
  const int nt = 1 << p.t;
  const int tstride = perm_tile_stride(nt);
  uint32_t* s_in = (uint32_t*)(tile + kPermBufs * tstride);
  uint32_t* s_out = s_in + nt;
  uint32_t* s_slot = s_out + nt;
  const int levels = perm_levels(p.n_rest);
  uint64_t* r_in = (uint64_t*)(((uintptr_t)(s_slot + nt) + 7) & ~(uintptr_t)7);   // [levels][256]
  uint64_t* r_out = r_in + 256 * levels;
  for (int i = threadIdx.x; i < nt; i += blockDim.x) {
    s_in[i] = __ldg(p.tab + i);
    s_out[i] = __ldg(p.tab + nt + i);
    s_slot[i] = (uint32_t)pad32((int)__ldg(p.tab + 2 * nt + i));
  }
  for (int e = threadIdx.x; e < 256 * levels; e += blockDim.x) {
    const int level = e >> 8, v = e & 255;
    uint64_t bi = 0, bo = 0;
    for (int k = 0; k < 8; ++k) {
      const int bit = level * 8 + k;
      if (bit < p.n_rest && ((v >> k) & 1)) {
        bi |= 1ULL << p.rest_in[bit];
        bo |= 1ULL << p.rest_out[bit];
      }
    }
    r_in[e] = bi;
    r_out[e] = bo;
  }
  __syncthreads();  // the tables are read below
  const uint64_t nrest_mask = (1ULL << p.n_rest) - 1;
  const uint64_t total_tiles = (uint64_t)p.P << p.n_rest;
  float2* __restrict__ out_lo = p.out + p.P * p.pstride;
  const float sc = (SPLIT == 3 || SPLIT == 6) ? pow2f(fp16_scale_exp(*p.scale)) : 1.0f;
  // input and output base offsets of tile blk: the pattern's stride plus the
  // rest bits of the tile index scattered through the per-byte tables
  auto tile_base = [&](uint64_t blk, int64_t& iofs, int64_t& dofs) {
    const uint64_t pp = blk >> p.n_rest, b = blk & nrest_mask;
    uint64_t bi = 0, bo = 0;
    for (int l = 0; l < levels; ++l) {
      const int v = (int)((b >> (8 * l)) & 255);
      bi |= r_in[256 * l + v];
      bo |= r_out[256 * l + v];
    }
    iofs = (int64_t)(pp * p.pstride + bi);
    dofs = (int64_t)(pp * p.pstride + bo);
  };
  // issue the copies of tile blk into buffer buf (an empty group past the
  // end keeps the group count uniform)
  auto issue = [&](uint64_t blk, int buf) {
    if (blk < total_tiles) {
      int64_t iofs, dofs;
      tile_base(blk, iofs, dofs);
      const float2* src = p.in + iofs;
      float2* dst = tile + buf * tstride;
      for (int i = threadIdx.x; i < nt; i += blockDim.x) cp_async8(dst + pad32(i), src + s_in[i]);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int k = 0; k < kPermBufs - 1; ++k) issue((uint64_t)blockIdx.x + (uint64_t)k * gridDim.x, k);
  int buf = 0;
  for (uint64_t blk = blockIdx.x; blk < total_tiles; blk += gridDim.x) {
    cp_async_wait<kPermBufs - 2>();   // this thread's copies of tile blk are done
    __syncthreads();                  // ... and everyone's; the buffer written out last round is free
    issue(blk + (uint64_t)(kPermBufs - 1) * gridDim.x, (buf + kPermBufs - 1) % kPermBufs);
    int64_t iofs, cur_dofs;
    tile_base(blk, iofs, cur_dofs);
    const float2* t = tile + buf * tstride;
    buf = (buf + 1) % kPermBufs;
    if (SPLIT < 4 && p.vec4) {
      // output bits 0 and 1 are tile bits 0 and 1: outputs 4g .. 4g + 3 of
      // the tile are consecutive in memory, from a 4-aligned index.  Fewer,
      // wider stores, but each warp's shared-memory reads take other tile
      // bits than in the loop below, so which is faster depends on the
      // permutation: a schedule variant of its own, chosen by timing.
      for (int g = threadIdx.x; g < (nt >> 2); g += blockDim.x) {
        const uint4 sl = *(const uint4*)(s_slot + 4 * g);
        const int64_t o = cur_dofs + s_out[4 * g];
        const float2 v0 = t[sl.x], v1 = t[sl.y], v2 = t[sl.z], v3 = t[sl.w];
        if (SPLIT == 1) {
          const float2 h0 = make_float2(tf32_rn(v0.x), tf32_rn(v0.y)), h1 = make_float2(tf32_rn(v1.x), tf32_rn(v1.y));
          const float2 h2 = make_float2(tf32_rn(v2.x), tf32_rn(v2.y)), h3 = make_float2(tf32_rn(v3.x), tf32_rn(v3.y));
          store4(p.out + o, h0, h1, h2, h3);
          store4(out_lo + o, make_float2(v0.x - h0.x, v0.y - h0.y), make_float2(v1.x - h1.x, v1.y - h1.y),
                 make_float2(v2.x - h2.x, v2.y - h2.y), make_float2(v3.x - h3.x, v3.y - h3.y));
        } else if (SPLIT == 3) {
          __half2* fh = (__half2*)p.out;
          __half2* fl = fh + p.P * p.pstride;
          __half2 h[4], l[4];
          const float2 v[4] = {v0, v1, v2, v3};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float2 w = make_float2(v[e].x * sc, v[e].y * sc);
            h[e] = __floats2half2_rn(w.x, w.y);
            const float2 hf = __half22float2(h[e]);
            l[e] = __floats2half2_rn(w.x - hf.x, w.y - hf.y);
          }
          store4(fh + o, h[0], h[1], h[2], h[3]);
          store4(fl + o, l[0], l[1], l[2], l[3]);
        } else if (SPLIT == 2) {
          __nv_bfloat162* bh = (__nv_bfloat162*)p.out;
          __nv_bfloat162* bl = bh + p.P * p.pstride;
          __nv_bfloat162 h[4], l[4];
          const float2 v[4] = {v0, v1, v2, v3};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            h[e] = __floats2bfloat162_rn(v[e].x, v[e].y);
            const float2 hf = __bfloat1622float2(h[e]);
            l[e] = __floats2bfloat162_rn(v[e].x - hf.x, v[e].y - hf.y);
          }
          store4(bh + o, h[0], h[1], h[2], h[3]);
          store4(bl + o, l[0], l[1], l[2], l[3]);
        } else {
          store4(p.out + o, v0, v1, v2, v3);
        }
      }
      continue;
    }
#pragma unroll 4
    for (int j = threadIdx.x; j < nt; j += blockDim.x) {
      const float2 v = t[s_slot[j]];
      const int64_t o = cur_dofs + s_out[j];
      if constexpr (SPLIT >= 4) {
        // the tensor-core B operand: output index o = k + K n of a pattern
        // becomes the 2 x 2 block [[re, -im], [im, re]] at pairs (2k, 2k+1)
        // of rows 2n and 2n + 1 of the [2N][2K] real embedding
        using PT = Pair<SPLIT - 4>;
        using T = typename PT::T;
        T* hi = (T*)p.out;
        T* lo = hi + 2 * p.P * p.pstride;
        const int64_t K = 1LL << p.embed_nk;
        const int64_t e0 = 2 * o - (o & (K - 1));
        T h, l;
        PT::split(v.x, -v.y, sc, h, l);
        hi[e0] = h;
        lo[e0] = l;
        PT::split(v.y, v.x, sc, h, l);
        hi[e0 + K] = h;
        lo[e0 + K] = l;
      } else if (SPLIT == 1) {
        const float2 h = make_float2(tf32_rn(v.x), tf32_rn(v.y));
        p.out[o] = h;
        out_lo[o] = make_float2(v.x - h.x, v.y - h.y);
      } else if (SPLIT == 3) {
        __half2* fh = (__half2*)p.out;
        __half2* fl = fh + p.P * p.pstride;
        const float2 w = make_float2(v.x * sc, v.y * sc);
        const __half2 h = __floats2half2_rn(w.x, w.y);
        const float2 hf = __half22float2(h);
        fh[o] = h;
        fl[o] = __floats2half2_rn(w.x - hf.x, w.y - hf.y);
      } else if (SPLIT == 2) {
        __nv_bfloat162* bh = (__nv_bfloat162*)p.out;
        __nv_bfloat162* bl = bh + p.P * p.pstride;
        const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
        const float2 hf = __bfloat1622float2(h);
        bh[o] = h;
        bl[o] = __floats2bfloat162_rn(v.x - hf.x, v.y - hf.y);
      } else {
        p.out[o] = v;
      }
    }
  }
  cp_async_wait<0>();
}

// Scale slot of the FP16x3 engine: max over the operand of |re| and |im|.
// Non-negative fp32 values order like their bit patterns, so the block maxima
// are merged with an unsigned atomicMax into the slot (zeroed before the pass).
__global__ void __launch_bounds__(256) k_absmax(AbsmaxParams p) {
  __shared__ float red[8];
  float m = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = __ldg(p.in + i);
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) atomicMax(p.out, __float_as_uint(m));
  }
}

cudaError_t launch_absmax(const AbsmaxParams& p, cudaStream_t s) {
  const int64_t grid = std::max<int64_t>(std::min<int64_t>((p.n + 255) / 256, (int64_t)kSMs * 8), 1);
  k_absmax<<<(unsigned)grid, 256, 0, s>>>(p);
  return cudaGetLastError();
}

// Largest dynamic shared memory of a permute launch: kPermBufs tiles of 2^10
// elements, the three 2^10-entry index tables and four levels of rest-bit
// tables (about 54 KB), above the 48 KB a launch gets without opting in.
static size_t perm_smem(int t, int n_rest) {
  const int nt = 1 << t;
  return sizeof(float2) * (size_t)kPermBufs * perm_tile_stride(nt) + 3 * sizeof(uint32_t) * (size_t)nt + 8 +
         2 * 256 * (size_t)perm_levels(n_rest) * sizeof(uint64_t);
}

cudaError_t prepare_permute() {
  const int mx = (int)perm_smem(10, 32);
  cudaError_t e = cudaFuncSetAttribute(k_permute<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_permute<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_permute<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_permute<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_permute<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_permute<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_permute<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  return e;
}

cudaError_t launch_permute(const PermParams& p, cudaStream_t s) {
  if (p.n_rest > 32) return cudaErrorInvalidValue;
  const int64_t blocks = (1LL << p.n_rest) * p.P;
  const int64_t grid = std::min<int64_t>(blocks, (int64_t)kSMs * 8);
  if (p.t < 0 || p.t > 10) return cudaErrorInvalidValue;
  const size_t smem = perm_smem(p.t, p.n_rest);
  if (p.split == 1) k_permute<1><<<(unsigned)grid, 256, smem, s>>>(p);
  else if (p.split == 2) k_permute<2><<<(unsigned)grid, 256, smem, s>>>(p);
  else if (p.split == 3) k_permute<3><<<(unsigned)grid, 256, smem, s>>>(p);
  else if (p.split == 4) k_permute<4><<<(unsigned)grid, 256, smem, s>>>(p);
  else if (p.split == 5) k_permute<5><<<(unsigned)grid, 256, smem, s>>>(p);
  else if (p.split == 6) k_permute<6><<<(unsigned)grid, 256, smem, s>>>(p);
  else k_permute<0><<<(unsigned)grid, 256, smem, s>>>(p);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ B prep
__global__ void k_bprep_c(BPrepParams p) {
  const int64_t K = 1LL << p.nk, N = 1LL << p.nn;
  const int64_t total = p.PB * K * N;
  float2* out = (float2*)p.out;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pb = e / (K * N), r = e % (K * N);
    const int64_t k = r / N, n = r % N;
    out[e] = p.B[pb * p.b_pstride + p.bk[k] + p.bn[n]];
  }
}

// Real embedding of B for C_r = A_r B_r with interleaved complex rows:
// Bt[j][i] (j = 2n + jc output column, i = 2k + ic reduction index) is
// [[re, -im], [im, re]] in (jc, ic); stored K-major as hi and lo planes in the
// GEMM engine's operand format (FMT 0: tf32-rounded fp32 hi + fp32 remainder;
// 1: bf16 hi + bf16 remainder; 2: fp16 of the value times the scale sc).  One
// thread per complex element of B: it writes the element's 2 x 2 block as two
// pairs of adjacent reals (rows 2n and 2n + 1) in each plane; consecutive
// threads take consecutive k, so every row segment is written contiguously.
// Its loads coalesce only when B's K legs are its low bits; otherwise the
// plan prepares B with the permute kernel in an embedding mode (split 4-6),
// which reads through a shared-memory tile.
template <int FMT>
__global__ void k_bprep_tc(BPrepParams p) {
  using T = typename Pair<FMT>::T;
  const int64_t K = 1LL << p.nk, N = 1LL << p.nn;
  const int64_t per = K * N;                  // complex elements per pattern
  const int64_t total = p.PB * per;
  T* hi = (T*)p.out;                          // pairs: [PB][2N][K] pairs of reals
  T* lo = hi + 2 * total;
  const float sc = FMT == 2 ? pow2f(fp16_scale_exp(*p.scale)) : 1.0f;
  // kU elements per thread and round, their loads issued before any store,
  // so that a grid of one block per SM (beside a running GEMM) still keeps
  // enough loads in flight
  constexpr int kU = 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e0 < total; e0 += kU * stride) {
    float2 b[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t e = e0 + u * stride;
      if (e < total) {
        const int64_t pb = e / per, r = e - pb * per;
        b[u] = p.B[pb * p.b_pstride + p.bk[r & (K - 1)] + p.bn[r >> p.nk]];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t e = e0 + u * stride;
      if (e >= total) break;
      const int64_t pb = e / per, r = e - pb * per;
      const int64_t n = r >> p.nk, k = r & (K - 1);
      const int64_t o0 = (pb * 2 * N + 2 * n) * K + k;   // pair (2k, 2k+1) of row 2n
      T h, l;
      Pair<FMT>::split(b[u].x, -b[u].y, sc, h, l);
      hi[o0] = h;
      lo[o0] = l;
      Pair<FMT>::split(b[u].y, b[u].x, sc, h, l);
      hi[o0 + K] = h;                                    // row 2n + 1
      lo[o0 + K] = l;
    }
  }
}

cudaError_t launch_bprep_c(const BPrepParams& p, cudaStream_t s) {
  const int64_t total = p.PB << (p.nk + p.nn);
  const int64_t grid = std::min<int64_t>((total + 255) / 256, (int64_t)kSMs * 8);
  k_bprep_c<<<(unsigned)std::max<int64_t>(grid, 1), 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_bprep_tc(const BPrepParams& p, cudaStream_t s, bool beside_gemm) {
  const int64_t total = p.PB << (p.nk + p.nn);
  // beside a running GEMM (one CTA per SM, most of the registers and shared
  // memory): one 256-thread block per SM, which fits next to it
  const int64_t cap = beside_gemm ? (int64_t)kSMs : (int64_t)kSMs * 16;
  const unsigned grid = (unsigned)std::max<int64_t>(std::min<int64_t>((total + 255) / 256, cap), 1);
  if (p.h16 == 2) k_bprep_tc<2><<<grid, 256, 0, s>>>(p);
  else if (p.h16 == 1) k_bprep_tc<1><<<grid, 256, 0, s>>>(p);
  else k_bprep_tc<0><<<grid, 256, 0, s>>>(p);
  return cudaGetLastError();
}

// ------------------------------------------------------------ SIMT GEMM
// Plain FP32 complex GEMM on CUDA cores: 64x64 complex tile, 16-deep k slab,
// 4x4 outputs per thread.  The reference "plain complex64" engine.
__global__ void __launch_bounds__(256) k_gemm_simt(GemmParams p) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ float2 As[BK][BM + 1];
  __shared__ float2 Bs[BK][BN];
  const int64_t tilesN = (p.N + BN - 1) / BN;
  const int64_t tm = blockIdx.x / tilesN, tn = blockIdx.x % tilesN;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const float2* __restrict__ Bg0 = (const float2*)p.B;
  for (int64_t pc = blockIdx.y; pc < p.PC; pc += gridDim.y) {
    const int64_t pa = map_p(p.mapA_mode, p.mapA, pc), pb = map_p(p.mapB_mode, p.mapB, pc);
    const float2* __restrict__ Ag = p.A + pa * p.M * p.K;
    const float2* __restrict__ Bg = Bg0 + pb * p.K * p.N;
    float2* __restrict__ Cg = p.C + pc * p.M * p.N;
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (int64_t k0 = 0; k0 < p.K; k0 += BK) {
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int e = tid + 256 * r;
        const int ml = e / BK, kl = e % BK;
        const int64_t m = tm * BM + ml, k = k0 + kl;
        As[kl][ml] = (m < p.M && k < p.K) ? __ldg(Ag + m * p.K + k) : make_float2(0.f, 0.f);
        const int kb = e / BN, nl = e % BN;
        const int64_t n = tn * BN + nl, kk = k0 + kb;
        Bs[kb][nl] = (n < p.N && kk < p.K) ? __ldg(Bg + kk * p.N + n) : make_float2(0.f, 0.f);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        float2 a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = cmul_add(acc[i][j], a[i], b[j]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t m = tm * BM + ty + 16 * i;
      if (m >= p.M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t n = tn * BN + tx + 16 * j;
        if (n < p.N) Cg[m * p.N + n] = acc[i][j];
      }
    }
  }
}

cudaError_t launch_gemm_simt(const GemmParams& p, cudaStream_t s) {
  const int64_t tiles = ((p.M + 63) / 64) * ((p.N + 63) / 64);
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  const int64_t gy = std::min<int64_t>(p.PC, 65535);
  k_gemm_simt<<<dim3((unsigned)tiles, (unsigned)gy), 256, 0, s>>>(p);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------- K4
// H[g][mu] += F[pidx[g]][open bits of mu]   (FP64 accumulation of slices)
__global__ void k_accum(AccumParams p) {
  const int64_t total = p.L << p.h;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = e >> p.h;
    const int64_t mu = e & ((1LL << p.h) - 1);
    int64_t off = (int64_t)__ldg(p.pidx + g) * p.f_pstride;
    for (int j = 0; j < p.h; ++j)
      if ((mu >> j) & 1) off |= 1LL << p.open_pos[j];
    const float2 v = __ldg(p.F + off);
    double2 hv = p.H[e];
    hv.x += (double)v.x;
    hv.y += (double)v.y;
    p.H[e] = hv;
  }
}

cudaError_t launch_accum(const AccumParams& p, cudaStream_t s) {
  const int64_t total = p.L << p.h;
  const int64_t grid = std::min<int64_t>((total + 255) / 256, (int64_t)kSMs * 8);
  k_accum<<<(unsigned)std::max<int64_t>(grid, 1), 256, 0, s>>>(p);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------- K7
// With seg_end (n_seg cumulative ends of merged requests), a missing key i of
// segment j records its index within the segment in status[j]; otherwise
// status[0] receives the smallest missing index.
__global__ void k_amplitudes(const double2* __restrict__ H, int h, const uint64_t* __restrict__ keys,
                             const uint32_t* __restrict__ groups, int64_t n_keys, uint64_t tail_mask,
                             const int* __restrict__ open_q, const uint64_t* __restrict__ bits, int64_t n, void* out,
                             int dtype, unsigned long long* status, const int64_t* __restrict__ seg_end, int n_seg) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t b = bits[i];
    const uint64_t key = b & tail_mask;
    int64_t lo = 0, hi = n_keys;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (keys[mid] < key) lo = mid + 1; else hi = mid;
    }
    double2 v = make_double2(0.0, 0.0);
    if (lo < n_keys && keys[lo] == key) {
      const int64_t g = groups[lo];
      int64_t mu = 0;
      for (int j = 0; j < h; ++j) mu |= (int64_t)((b >> open_q[j]) & 1ULL) << j;
      v = H[(g << h) + mu];
    } else if (seg_end) {
      int j = 0;
      while (j < n_seg - 1 && i >= seg_end[j]) ++j;
      atomicMin(status + j, (unsigned long long)(i - (j ? seg_end[j - 1] : 0)));
    } else {
      atomicMin(status, (unsigned long long)i);
    }
    if (dtype == 1) ((double2*)out)[i] = v;
    else ((float2*)out)[i] = make_float2((float)v.x, (float)v.y);
  }
}

cudaError_t launch_amplitudes(const double2* H, int h, const uint64_t* keys, const uint32_t* groups, int64_t n_keys,
                              uint64_t tail_mask, const int* open_q, const uint64_t* bits, int64_t n, void* out,
                              int dtype, unsigned long long* status, cudaStream_t s, const int64_t* seg_end,
                              int n_seg) {
  if (n <= 0) return cudaSuccess;
  const int64_t grid = std::min<int64_t>((n + 255) / 256, (int64_t)kSMs * 8);
  k_amplitudes<<<(unsigned)grid, 256, 0, s>>>(H, h, keys, groups, n_keys, tail_mask, open_q, bits, n, out, dtype,
                                              status, seg_end, n_seg);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------- K5
// One warp per group: chunks of 32 members, each chunk reduced by an inclusive
// warp scan whose last lane is added to a running carry.  The sampler repeats
// exactly this order, so its prefix sums end at the same Z[g].
__device__ __forceinline__ double warp_inclusive_scan(double v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const double u = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += u;
  }
  return v;
}

__global__ void k_group_norms(const double2* __restrict__ H, int64_t L, int h, double* __restrict__ Z) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t l = 1LL << h;
  for (int64_t g = warp; g < L; g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    double carry = 0.0;
    for (int64_t c = 0; c < l; c += 32) {
      double w = 0.0;
      if (c + lane < l) {
        const double2 v = H[(g << h) + c + lane];
        w = v.x * v.x + v.y * v.y;
      }
      const double s = warp_inclusive_scan(w);
      carry += __shfl_sync(0xffffffffu, s, 31);
    }
    if (lane == 0) Z[g] = carry;
  }
}

// Deterministic single-block sum of Z into N.
__global__ void k_sum(const double* __restrict__ Z, int64_t L, double* N) {
  __shared__ double part[32];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < L; i += blockDim.x) acc += Z[i];
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    if (threadIdx.x == 0) *N = v;
  }
}

// XEB reductions (FP64): part[b] = sum |a_i|^2 and part[nb + b] = sum log |a_i|^2
// over block b's share of the n amplitudes (grid-stride, then a block tree).
__global__ void __launch_bounds__(256) k_xeb_partial(const double2* __restrict__ a, int64_t n, double* part) {
  __shared__ double s1[8], s2[8];
  double p = 0.0, lp = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = a[i];
    const double w = v.x * v.x + v.y * v.y;
    p += w;
    lp += log(w);
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    p += __shfl_xor_sync(0xffffffffu, p, d);
    lp += __shfl_xor_sync(0xffffffffu, lp, d);
  }
  if ((threadIdx.x & 31) == 0) {
    s1[threadIdx.x >> 5] = p;
    s2[threadIdx.x >> 5] = lp;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t1 = 0.0, t2 = 0.0;
    for (int w = 0; w < 8; ++w) {
      t1 += s1[w];
      t2 += s2[w];
    }
    part[blockIdx.x] = t1;
    part[gridDim.x + blockIdx.x] = t2;
  }
}

cudaError_t launch_xeb_sums(const double2* amp, int64_t n, double* part, double* sums, cudaStream_t s) {
  const int64_t nb = std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)kSMs * 4));
  k_xeb_partial<<<(unsigned)nb, 256, 0, s>>>(amp, n, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sum<<<1, 1024, 0, s>>>(part, nb, sums);
  k_sum<<<1, 1024, 0, s>>>(part + nb, nb, sums + 1);
  return cudaGetLastError();
}

int64_t xeb_partials(int64_t n) { return 2 * std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)kSMs * 4)); }

cudaError_t launch_group_norms(const double2* H, int64_t L, int h, double* Z, double* N, cudaStream_t s) {
  const int64_t warps = L;
  const int64_t grid = std::min<int64_t>((warps * 32 + 255) / 256, (int64_t)kSMs * 8);
  k_group_norms<<<(unsigned)std::max<int64_t>(grid, 1), 256, 0, s>>>(H, L, h, Z);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (N) {
    k_sum<<<1, 1024, 0, s>>>(Z, L, N);
    e = cudaGetLastError();
  }
  return e;
}

// ---------------------------------------------------------------------- K6
// Philox-4x32-10 (Salmon et al., SC'11): multipliers 0xD2511F53, 0xCD9E8D57,
// Weyl key increments 0x9E3779B9, 0xBB67AE85, ten rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    if (r != 9) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
  }
  return c;
}

__device__ __forceinline__ double u53(uint32_t lo, uint32_t hi) {
  const uint64_t x = ((uint64_t)hi << 32) | lo;
  return (double)(x >> 11) * 0x1.0p-53;
}

// |h|^2 with each operation rounded to nearest (no fused multiply-add), so
// that weights and the comparisons built on them are reproducible bit by bit.
__device__ __forceinline__ double weight_rn(double2 v) { return __dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y)); }

// One warp per sample, group i mod L.
//   method 0: exact draw by inverse CDF over the chunked warp-scan prefix sums
//             of |H[g][mu]|^2 (same order as k_group_norms);
//   method 1: Metropolis chain with uniform proposals (the paper's in-group
//             MCMC, Method and Supplement): start at member 0; for t < T,
//             propose mu' = bits of Philox(i, 2, t), accept when
//             u * w(mu) < w(mu');
//   method 2: frugal rejection sampling (Supplement, bitstring choice): for
//             t < 64 M rounds, draw mu = bits of Philox(i, 3, t) and accept
//             when (u * M) * Z < w(mu) * l; after the last round keep mu.
__global__ void k_sample(SampleParams p) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t l = 1LL << p.h;
  const uint2 key = make_uint2((uint32_t)p.seed, (uint32_t)(p.seed >> 32));
  const uint64_t full = p.n_qubits >= 64 ? ~0ULL : ((1ULL << p.n_qubits) - 1);
  for (int64_t i = warp; i < p.n; i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t g = i % p.L;
    const uint32_t ilo = (uint32_t)i, ihi = (uint32_t)((uint64_t)i >> 32);
    const uint4 r = philox4x32_10(make_uint4(ilo, ihi, 0u, 0u), key);
    const double u_mix = u53(r.x, r.y), u_pick = u53(r.z, r.w);
    if (p.mix > 0.0 && u_mix < p.mix) {
      const uint4 q = philox4x32_10(make_uint4(ilo, ihi, 1u, 0u), key);
      if (lane == 0) p.out[i] = ((((uint64_t)q.y) << 32) | q.x) & full;
      continue;
    }
    const double2* __restrict__ Hg = p.H + (g << p.h);
    int64_t mu = l - 1;
    if (p.method == 1) {
      // lane 0 runs the chain (it is sequential); the other lanes idle
      if (lane == 0) {
        int64_t cur = 0;
        double wc = weight_rn(Hg[0]);
        for (int64_t t = 0; t < p.param; ++t) {
          const uint4 q = philox4x32_10(make_uint4(ilo, ihi, 2u, (uint32_t)t), key);
          const int64_t prop = (int64_t)(q.x & (uint32_t)(l - 1));
          const double wp = weight_rn(Hg[prop]);
          const double u = u53(q.z, q.w);
          if (__dmul_rn(u, wc) < wp) { cur = prop; wc = wp; }
        }
        mu = cur;
      }
    } else {
      // chunked warp-scan total (exact draw and frugal bound)
      double Z = 0.0;
      for (int64_t c = 0; c < l; c += 32) {
        const double w = (c + lane < l) ? weight_rn(Hg[c + lane]) : 0.0;
        const double s = warp_inclusive_scan(w);
        Z += __shfl_sync(0xffffffffu, s, 31);
      }
      if (p.method == 2) {
        if (lane == 0) {
          const double M = (double)p.param;
          const double bound = __dmul_rn(M, Z);
          int64_t cand = 0;
          for (int64_t t = 0; t < 64 * p.param; ++t) {
            const uint4 q = philox4x32_10(make_uint4(ilo, ihi, 3u, (uint32_t)t), key);
            cand = (int64_t)(q.x & (uint32_t)(l - 1));
            const double u = u53(q.z, q.w);
            if (__dmul_rn(u, bound) < __dmul_rn(weight_rn(Hg[cand]), (double)l)) break;
          }
          mu = cand;
        }
      } else if (Z > 0.0) {
        const double t = u_pick * Z;
        double carry = 0.0;
        for (int64_t c = 0; c < l; c += 32) {
          const double w = (c + lane < l) ? weight_rn(Hg[c + lane]) : 0.0;
          const double s = warp_inclusive_scan(w);
          const bool hit = (c + lane < l) && (carry + s > t);
          const unsigned ball = __ballot_sync(0xffffffffu, hit);
          if (ball) { mu = c + __ffs(ball) - 1; break; }
          carry += __shfl_sync(0xffffffffu, s, 31);
        }
      } else {
        mu = (int64_t)(u_pick * (double)l);
        if (mu >= l) mu = l - 1;
      }
    }
    if (lane == 0) {
      uint64_t s = p.tails[g] & ~p.open_mask;
      for (int j = 0; j < p.h; ++j) s |= (uint64_t)((mu >> j) & 1) << p.open_q[j];
      p.out[i] = s;
    }
  }
}

cudaError_t launch_sample(const SampleParams& p, cudaStream_t s) {
  if (p.n <= 0) return cudaSuccess;
  const int64_t grid = std::min<int64_t>((p.n * 32 + 255) / 256, (int64_t)kSMs * 16);
  k_sample<<<(unsigned)grid, 256, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace tn
