// The learned MPPI proposal: a 3-layer MLP (in -> hidden -> hidden -> out, GELU) trained and
// evaluated with BF16 operands and FP32 accumulation on the 5th-generation tensor cores.
//
// GEMM D[M x N] = A[M x K] . B[N x K]^T (both K-major BF16): per CTA a 128 x BN tile, TMA loads
// of 128B-swizzled 64-wide K slices into a 4-stage shared-memory ring (mbarrier handshakes),
// one thread issues tcgen05.mma (kind::f16, M=128, N=BN, K=16 per instruction) into a TMEM
// accumulator, and four warps run the fused epilogue from tcgen05.ld (bias, GELU or its
// derivative, BF16/FP32 stores).  Every mbarrier wait is bounded: a wait that gives up sets the
// error word, the CTA skips its remaining work, frees its TMEM and returns.
#include <atomic>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>

#include "comfree.h"
#include "cf_internal.cuh"

namespace cf {
namespace mlp {

// Two stages of the TMA ring: the products here run at most four BK steps per CTA (K = 64 or
// 256, split-K slices of the batch), which two buffers already overlap, and 65 KB of shared
// memory per 128-wide CTA lets three CTAs share an SM (a 4-stage ring of 129 KB allowed one:
// the 256- to 1024-CTA grids then ran in several waves)
constexpr int BM = 128, BK = 64, STAGES = 2;
constexpr uint32_t kWaitLimit = 1u << 22;

enum Epi { EPI_BIAS_GELU = 0, EPI_BIAS_F32 = 1, EPI_F32 = 2, EPI_GELU_BWD = 3 };

struct EpiArgs {
  const float* bias;        // [N] (EPI_BIAS_*)
  __nv_bfloat16* out_bf16;  // [M x ldo] activations (GELU) or gradients (GELU_BWD)
  __nv_bfloat16* out_z;     // [M x ldo] pre-activation (EPI_BIAS_GELU)
  const __nv_bfloat16* z;   // [M x ldo] pre-activation read by EPI_GELU_BWD
  float* out_f32;           // [M x ldo] (EPI_BIAS_F32, EPI_F32)
  size_t slice_stride;      // split-K: CTA z stores its partial tile at out_f32 + z * slice_stride
  int ldo;
  int m_valid;              // rows >= m_valid are not stored
  int* err;
  __nv_bfloat16* out_t;     // optional [N x ldt] transposed copy of out_bf16 (EPI_BIAS_GELU, EPI_GELU_BWD)
  int ldt;
  float* colsum;            // optional with out_t, EPI_GELU_BWD: [M / 128 x ldo] column sums of out_bf16
                            // over each CTA's 128 rows (the bias gradient's partial sums)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// bounded wait on the phase with the given parity; false = gave up
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t addr = smem_u32(bar);
  for (uint32_t i = 0; i < kWaitLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused by swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // descriptor version
  d |= (uint64_t)2 << 61;              // 128B swizzle
  return d;
}

// instruction descriptor, kind::f16: FP32 accumulate, BF16 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// The epilogue's shared memory, behind the idle operand ring: per warp a [32][20] float slice,
// then per warp a [32][kEpiTB] bf16 copy of the slice's outputs, then [4][BN] column sums.
constexpr int kEpiTB = 18;
__device__ __forceinline__ float* epi_colsum_smem(uint8_t* smem) {
  return reinterpret_cast<float*>(smem) + 4 * 32 * 20 + 4 * 32 * kEpiTB / 2;
}

// TR: also write the transposed copy ep.out_t (EPI_BIAS_GELU, EPI_GELU_BWD); a template
// parameter, so that the instantiations without it keep the plain epilogue's code
template <int BN, int EPI, bool TR = false>
__global__ void __launch_bounds__(128) gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                   const __grid_constant__ CUtensorMap tmB, EpiArgs ep, int K) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
  __shared__ uint32_t tmem_base;
  __shared__ int s_ok;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int nk = K / BK;              // K: this CTA's share of the reduction (split-K: blockIdx.z)
  const int kz = blockIdx.z * K;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    mbar_init(&done, 1);
    s_ok = 1;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = idesc_bf16(BM, BN);

  if (threadIdx.x == 0) {
    bool ok = true;
    // bit s of `pending`: stage s has a load in flight (a stage holds at most one); bit s of
    // `phase`: the parity of the loads consumed from stage s, i.e. of the phase to wait on next
    unsigned pending = 0, phase = 0;
    const int pre = nk < STAGES ? nk : STAGES;
    for (int s = 0; s < pre; ++s) {
      mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
      tma_load_2d(sA + s * A_BYTES, &tmA, kz + s * BK, m0, &full[s]);
      tma_load_2d(sB + s * B_BYTES, &tmB, kz + s * BK, n0, &full[s]);
      pending |= 1u << s;
    }
    for (int k = 0; k < nk && ok; ++k) {
      const int s = k % STAGES;
      const uint32_t par = (k / STAGES) & 1;
      if (!mbar_wait(&full[s], par)) { ok = false; break; }
      pending &= ~(1u << s);
      phase ^= 1u << s;
      tc_fence_after();
      const uint64_t da = smem_desc(smem_u32(sA + s * A_BYTES));
      const uint64_t db = smem_desc(smem_u32(sB + s * B_BYTES));
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk)
        umma_bf16(tmem, da + 2 * kk, db + 2 * kk, idesc, (k | kk) ? 1u : 0u);
      umma_commit(&empty[s]);
      if (k + STAGES < nk) {
        if (!mbar_wait(&empty[s], par)) { ok = false; break; }
        mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
        tma_load_2d(sA + s * A_BYTES, &tmA, kz + (k + STAGES) * BK, m0, &full[s]);
        tma_load_2d(sB + s * B_BYTES, &tmB, kz + (k + STAGES) * BK, n0, &full[s]);
        pending |= 1u << s;
      }
    }
    if (!ok) {
      // a wait gave up: flag it, then let this CTA's own loads in flight land (each wait again
      // bounded) before the shared memory they write is released
      s_ok = 0;
      atomicOr(ep.err, CF_FLAG_TIMEOUT);
      for (int s = 0; s < STAGES; ++s)
        if ((pending >> s) & 1u) mbar_wait(&full[s], (phase >> s) & 1u);
    }
    // `done` fires once every MMA issued here has completed, so TMEM is freed only after them
    umma_commit(&done);
  }
  __syncwarp();
  bool ok = mbar_wait(&done, 0);
  tc_fence_after();
  if (!ok && lane == 0) atomicOr(ep.err, CF_FLAG_TIMEOUT);
  if (ok && s_ok) {
    // tcgen05.ld hands each lane one row; a 32-row x 16-column slice is staged in shared memory
    // (the operand ring is idle once `done` has fired) and written back four columns per lane,
    // four lanes per row and eight rows per instruction, so that global stores (and the loads
    // of z) are 16- or 8-byte vectors on contiguous 64- or 32-byte row segments.  Row stride 20
    // floats keeps the staging writes of a quarter-warp on distinct banks.
    float* stage = reinterpret_cast<float*>(smem) + warp * (32 * 20);
    // the slice's bf16 outputs again, for the optional transposed copy: rows of kTB = 18
    // elements (4-byte aligned; the two half-columns a lane pair reads fall on different banks)
    constexpr bool trans = TR && (EPI == EPI_BIAS_GELU || EPI == EPI_GELU_BWD);
    constexpr int kTB = kEpiTB;
    __nv_bfloat16* tstage = reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<float*>(smem) + 4 * 32 * 20) +
                            warp * (32 * kTB);
    float* csm = epi_colsum_smem(smem);
    const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
    const int quad = lane & 3, ro = lane >> 2;
    float* out_f32 = ep.out_f32 + (size_t)blockIdx.z * ep.slice_stride;
    for (int c = 0; c < BN; c += 16) {
      float v[16];
      tmem_ld16(tbase + c, v);
#pragma unroll
      for (int i = 0; i < 16; i += 4)
        *reinterpret_cast<float4*>(stage + lane * 20 + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
      __syncwarp();
      const int n = n0 + c + 4 * quad;
      float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
      if (EPI == EPI_BIAS_GELU || EPI == EPI_BIAS_F32) b = *reinterpret_cast<const float4*>(ep.bias + n);
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        const int r = 8 * rr + ro;
        const int row = m0 + warp * 32 + r;
        if (row < ep.m_valid) {
          const float4 a = *reinterpret_cast<const float4*>(stage + r * 20 + 4 * quad);
          const size_t o = (size_t)row * ep.ldo + n;
          if (EPI == EPI_BIAS_GELU) {
            const float z0 = a.x + b.x, z1 = a.y + b.y, z2 = a.z + b.z, z3 = a.w + b.w;
            __nv_bfloat162 zz[2] = {__floats2bfloat162_rn(z0, z1), __floats2bfloat162_rn(z2, z3)};
            __nv_bfloat162 hh[2] = {__floats2bfloat162_rn(gelu(z0), gelu(z1)), __floats2bfloat162_rn(gelu(z2), gelu(z3))};
            *reinterpret_cast<uint2*>(ep.out_z + o) = *reinterpret_cast<const uint2*>(zz);
            *reinterpret_cast<uint2*>(ep.out_bf16 + o) = *reinterpret_cast<const uint2*>(hh);
            if (trans) {
              __nv_bfloat162* t2 = reinterpret_cast<__nv_bfloat162*>(tstage + r * kTB + 4 * quad);
              t2[0] = hh[0];
              t2[1] = hh[1];
            }
          } else if (EPI == EPI_BIAS_F32) {
            *reinterpret_cast<float4*>(out_f32 + o) = make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
          } else if (EPI == EPI_F32) {
            *reinterpret_cast<float4*>(out_f32 + o) = a;
          } else {
            const uint2 zr = *reinterpret_cast<const uint2*>(ep.z + o);
            const __nv_bfloat162* zp = reinterpret_cast<const __nv_bfloat162*>(&zr);
            __nv_bfloat162 gg[2] = {
                __floats2bfloat162_rn(a.x * gelu_grad(__low2float(zp[0])), a.y * gelu_grad(__high2float(zp[0]))),
                __floats2bfloat162_rn(a.z * gelu_grad(__low2float(zp[1])), a.w * gelu_grad(__high2float(zp[1])))};
            *reinterpret_cast<uint2*>(ep.out_bf16 + o) = *reinterpret_cast<const uint2*>(gg);
            if (trans) {
              __nv_bfloat162* t2 = reinterpret_cast<__nv_bfloat162*>(tstage + r * kTB + 4 * quad);
              t2[0] = gg[0];
              t2[1] = gg[1];
            }
          }
        }
      }
      __syncwarp();
      if (trans) {
        // transposed copy: lane pair (2j, 2j + 1) writes column n0 + c + j, rows 16h .. 16h + 15 of
        // this warp's 32 as two 16-byte vectors (ldt is a multiple of 16 elements)
        const int j = lane >> 1, h = lane & 1;
        const int row0 = m0 + warp * 32 + 16 * h;
        __nv_bfloat16* dst = ep.out_t + (size_t)(n0 + c + j) * ep.ldt + row0;
        const __nv_bfloat16* src = tstage + 16 * h * kTB + j;
        float csum = 0.f;  // this half-column's stored values, summed in row order
        if (row0 + 16 <= ep.m_valid) {
          uint32_t w[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const __nv_bfloat16 lo = src[(2 * k) * kTB], hi = src[(2 * k + 1) * kTB];
            w[k] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
            csum += __bfloat162float(lo);
            csum += __bfloat162float(hi);
          }
          reinterpret_cast<uint4*>(dst)[0] = make_uint4(w[0], w[1], w[2], w[3]);
          reinterpret_cast<uint4*>(dst)[1] = make_uint4(w[4], w[5], w[6], w[7]);
        } else {
          for (int t = 0; t < 16; ++t)
            if (row0 + t < ep.m_valid) {
              dst[t] = src[t * kTB];
              csum += __bfloat162float(src[t * kTB]);
            }
        }
        if (EPI == EPI_GELU_BWD && ep.colsum != nullptr) {
          // both halves of the column (lanes 2j, 2j + 1), kept per warp until the CTA's barrier
          csum += __shfl_xor_sync(0xffffffffu, csum, 1);
          if (h == 0) csm[warp * BN + c + j] = csum;
        }
        __syncwarp();
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
  if (TR && EPI == EPI_GELU_BWD && ep.colsum != nullptr && s_ok && warp == 0) {
    // the four warps' column sums of this CTA's 128 rows, added in warp order
    const float* csm = epi_colsum_smem(smem);
    for (int col = lane; col < BN; col += 32)
      ep.colsum[(size_t)blockIdx.y * ep.ldo + n0 + col] = ((csm[col] + csm[BN + col]) + csm[2 * BN + col]) + csm[3 * BN + col];
  }
}

// ---------------------------------------------------------------------------------------
// elementwise kernels
// ---------------------------------------------------------------------------------------
// features [B x fin] fp32 -> [Bp x kin] bf16, zero padded in both directions
__global__ void pack_input(const float* x, int B, int fin, int Bp, int kin, __nv_bfloat16* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Bp * kin) return;
  int r = i / kin, c = i % kin;
  out[i] = __float2bfloat16_rn(r < B && c < fin ? x[(size_t)r * fin + c] : 0.f);
}

// out[c][r] = in[r][c] for a [R x C] bf16 matrix (32 x 32 tiles through shared memory)
// out[C x R] = in[R x C]^T by 64 x 64 tiles of a (32, 8) block: each lane moves two adjacent
// elements, so a warp reads and writes 128-byte row segments (bf16 pairs when the row length is
// even, single elements at odd edges); rows of 65 elements in shared memory keep the column
// reads of a warp on distinct banks
__global__ void transpose_bf16(const __nv_bfloat16* in, int R, int C, __nv_bfloat16* out) {
  __shared__ __nv_bfloat16 t[64][65];
  const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64, x2 = 2 * threadIdx.x;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  for (int k = threadIdx.y; k < 64; k += blockDim.y) {
    const int r = r0 + k, c = c0 + x2;
    __nv_bfloat16 a = zero, b = zero;
    if (r < R) {
      const __nv_bfloat16* src = in + (size_t)r * C + c;
      if ((C & 1) == 0 && c + 1 < C) {
        const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(src);
        a = v.x;
        b = v.y;
      } else {
        if (c < C) a = src[0];
        if (c + 1 < C) b = src[1];
      }
    }
    t[k][x2] = a;
    t[k][x2 + 1] = b;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 64; k += blockDim.y) {
    const int c = c0 + k, r = r0 + x2;
    if (c >= C) continue;
    __nv_bfloat16* dst = out + (size_t)c * R + r;
    if ((R & 1) == 0 && r + 1 < R) {
      __nv_bfloat162 v;
      v.x = t[x2][k];
      v.y = t[x2 + 1][k];
      *reinterpret_cast<__nv_bfloat162*>(dst) = v;
    } else {
      if (r < R) dst[0] = t[x2][k];
      if (r + 1 < R) dst[1] = t[x2 + 1][k];
    }
  }
}

// Gaussian negative log-likelihood of targets a under mean mu = y[:, :D] and log-std
// s = clamp(y[:, D:], lo, hi):  l = sum_d ((a - mu)^2 / (2 e^{2s}) + s) / (B D).
// Writes dL/dy as bf16 twice: dy [Bp x 2D] (zero rows past B) for the backward product through
// W3, and its transpose dyt [2D x Bp] for the weight gradient, both with coalesced stores.  A
// (32, 8) block takes 64 rows x 64 columns of mu (and the same 64 columns of s): each lane
// computes two adjacent columns of a row, the tile goes through shared memory (rows of 65
// elements, so that the column reads of a warp fall on distinct banks) and is written
// transposed as bf16 pairs.  The loss is reduced per block (shuffles, then shared memory) and
// added with one atomic per block.  The bias gradient's partial sums: each block also writes
// the column sums of its 64 rows of the stored (bf16) dL/dy into part[Bp / 64][2D], adding its
// 8 row groups in order.  D and Bp are multiples of 64.
__global__ void __launch_bounds__(256) nll_grad(const float* y, const float* a, int B, int Bp, int D, float lo, float hi,
                                                __nv_bfloat16* dy, __nv_bfloat16* dyt, float* loss, float* part) {
  __shared__ __nv_bfloat16 tm[64][65], ts[64][65];
  __shared__ float red[8];
  __shared__ float4 csum[8][32];
  float4 cs = make_float4(0.f, 0.f, 0.f, 0.f);  // this thread's two mu columns, then two s columns
  const int r0 = blockIdx.y * 64, d0 = blockIdx.x * 64, x2 = 2 * threadIdx.x;
  const float inv_n = 1.f / ((float)B * (float)D);
  float l = 0.f;
  for (int k = threadIdx.y; k < 64; k += blockDim.y) {
    const int r = r0 + k, d = d0 + x2;
    float gm[2] = {0.f, 0.f}, gs[2] = {0.f, 0.f};
    if (r < B) {
      const float2 mu = *reinterpret_cast<const float2*>(y + (size_t)r * 2 * D + d);
      const float2 sr = *reinterpret_cast<const float2*>(y + (size_t)r * 2 * D + D + d);
      const float* ar = a + (size_t)r * D + d;  // the caller's targets: no alignment assumed
      const float m2[2] = {mu.x, mu.y}, s2[2] = {sr.x, sr.y}, a2[2] = {ar[0], ar[1]};
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const float s = fminf(fmaxf(s2[i], lo), hi);
        const float e = a2[i] - m2[i];
        const float iv = expf(-2.f * s);
        l += (0.5f * e * e * iv + s) * inv_n;
        gm[i] = -e * iv * inv_n;
        gs[i] = (s2[i] > lo && s2[i] < hi) ? (1.f - e * e * iv) * inv_n : 0.f;
      }
    }
    const __nv_bfloat162 bm = __floats2bfloat162_rn(gm[0], gm[1]), bs = __floats2bfloat162_rn(gs[0], gs[1]);
    *reinterpret_cast<__nv_bfloat162*>(dy + (size_t)r * 2 * D + d) = bm;
    *reinterpret_cast<__nv_bfloat162*>(dy + (size_t)r * 2 * D + D + d) = bs;
    cs.x += __low2float(bm);
    cs.y += __high2float(bm);
    cs.z += __low2float(bs);
    cs.w += __high2float(bs);
    tm[k][x2] = bm.x;
    tm[k][x2 + 1] = bm.y;
    ts[k][x2] = bs.x;
    ts[k][x2 + 1] = bs.y;
  }
  csum[threadIdx.y][threadIdx.x] = cs;
  __syncthreads();
  if (threadIdx.y == 0) {
    float4 t = csum[0][threadIdx.x];
    for (int g = 1; g < 8; ++g) {
      const float4 u = csum[g][threadIdx.x];
      t.x += u.x; t.y += u.y; t.z += u.z; t.w += u.w;
    }
    float* pr = part + (size_t)blockIdx.y * 2 * D;
    pr[d0 + x2] = t.x;
    pr[d0 + x2 + 1] = t.y;
    pr[D + d0 + x2] = t.z;
    pr[D + d0 + x2 + 1] = t.w;
  }
  for (int k = threadIdx.y; k < 64; k += blockDim.y) {
    const int r = r0 + x2;
    __nv_bfloat162 vm, vs;
    vm.x = tm[x2][k];
    vm.y = tm[x2 + 1][k];
    vs.x = ts[x2][k];
    vs.y = ts[x2 + 1][k];
    *reinterpret_cast<__nv_bfloat162*>(dyt + (size_t)(d0 + k) * Bp + r) = vm;
    *reinterpret_cast<__nv_bfloat162*>(dyt + (size_t)(D + d0 + k) * Bp + r) = vs;
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
  const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
  if ((threadIdx.x & 31) == 0) red[warp] = l;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x * blockDim.y >> 5); ++w) t += red[w];
    if (t != 0.f) atomicAdd(loss, t);
  }
}

// Bias gradients db[n] = sum over the partial sums part[k][n], k = 0 .. slices - 1, in a fixed
// order (deterministic); the partials are written by nll_grad (one per 64-row tile) and by the
// GELU-derivative GEMM epilogues (one per 128-row CTA).  N is a multiple of 64.
__global__ void __launch_bounds__(256) bias_grad_final(const float* part, int N, int slices, float* db) {
  // 64 columns per block, two adjacent ones per lane; warp w adds partials w, w + 8, ... in
  // order, then warp 0 adds the 8 warps' sums in order
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c0 = blockIdx.x * 64 + 2 * lane;
  float2 t = make_float2(0.f, 0.f);
  for (int k = warp; k < slices; k += 8) {
    const float2 v = *reinterpret_cast<const float2*>(part + (size_t)k * N + c0);
    t.x += v.x;
    t.y += v.y;
  }
  __shared__ float2 red[8][32];
  red[warp][lane] = t;
  __syncthreads();
  if (warp == 0) {
    float2 u = red[0][lane];
    for (int w = 1; w < 8; ++w) { u.x += red[w][lane].x; u.y += red[w][lane].y; }
    db[c0] = u.x;
    db[c0 + 1] = u.y;
  }
}

// Adam on the fp32 master weights; refreshes the bf16 copy (and its transpose when given)
__global__ void adam(float* w, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps, float c1,
                     float c2, __nv_bfloat16* wb, __nv_bfloat16* wt, int rows, int cols) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  if (wb) wb[i] = __float2bfloat16_rn(wi);
  if (wt) {
    int r = i / cols, c = i % cols;
    wt[(size_t)c * rows + r] = __float2bfloat16_rn(wi);
  }
}

__global__ void to_bf16(const float* w, int n, __nv_bfloat16* wb, __nv_bfloat16* wt, int rows, int cols) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  wb[i] = __float2bfloat16_rn(w[i]);
  if (wt) {
    int r = i / cols, c = i % cols;
    wt[(size_t)c * rows + r] = __float2bfloat16_rn(w[i]);
  }
}

}  // namespace mlp
}  // namespace cf

// =======================================================================================
// host side
// =======================================================================================
using namespace cf::mlp;

namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;
cf_status mfail(cf_status s, const char* msg) {
  cf::set_last_error(msg);
  return s;
}

bool get_encoder() {
  if (g_encode) return true;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return false;
  g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  return true;
}

// 2D bf16 tensor map of a row-major [rows x cols] matrix, box = 64 columns x box_rows rows
bool make_map(CUtensorMap* m, const void* ptr, int rows, int cols, int box_rows) {
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t gemm_smem(int BN) { return (size_t)STAGES * (BM * BK * 2 + BN * BK * 2) + 1024; }

template <int BN, int EPI, bool TR = false>
cudaError_t gemm_launch(const void* A, int M, const void* B, int N, int K, const EpiArgs& ep, cudaStream_t s,
                        int split = 1) {
  CUtensorMap ta, tb;
  if (!make_map(&ta, A, M, K, BM) || !make_map(&tb, B, N, K, BN)) return cudaErrorInvalidValue;
  if (TR && (ep.out_t == nullptr || ep.ldt % 16 || ep.ldt < M)) return cudaErrorInvalidValue;
  // the dynamic shared memory opt-in is per device: one bit per device that has it
  static std::atomic<uint64_t> attr{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!((attr.load() >> dev) & 1u)) {
    e = cudaFuncSetAttribute(gemm_kernel<BN, EPI, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)gemm_smem(BN));
    if (e != cudaSuccess) return e;
    attr.fetch_or(uint64_t(1) << dev);
  }
  dim3 grid(N / BN, M / BM, split);
  gemm_kernel<BN, EPI, TR><<<grid, 128, gemm_smem(BN), s>>>(ta, tb, ep, K / split);
  return cudaGetLastError();
}

// ep.out_t set: the epilogue also writes the transposed copy (EPI_BIAS_GELU, EPI_GELU_BWD)
template <int EPI>
cudaError_t gemm(const void* A, int M, const void* B, int N, int K, const EpiArgs& ep, cudaStream_t s) {
  if (M % BM || K % BK || N % 64) return cudaErrorInvalidValue;
  constexpr bool can_t = EPI == EPI_BIAS_GELU || EPI == EPI_GELU_BWD;
  if (ep.out_t && !can_t) return cudaErrorInvalidValue;
  if (ep.colsum && (EPI != EPI_GELU_BWD || !ep.out_t || ep.ldo != N)) return cudaErrorInvalidValue;
  if (can_t && ep.out_t)
    return N % 128 == 0 ? gemm_launch<128, EPI, can_t>(A, M, B, N, K, ep, s) : gemm_launch<64, EPI, can_t>(A, M, B, N, K, ep, s);
  if (N % 128 == 0) return gemm_launch<128, EPI>(A, M, B, N, K, ep, s);
  return gemm_launch<64, EPI>(A, M, B, N, K, ep, s);
}

// out[i] = sum_z part[z * n + i], the split-K partial tiles added in order
__global__ void splitk_reduce(const float* part, int split, size_t n, float* out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float t = 0.f;
    for (int z = 0; z < split; ++z) t += part[(size_t)z * n + i];
    out[i] = t;
  }
}

constexpr int kMaxSplit = 64;     // slices of one split-K product
constexpr int kSplitScratch = 16; // scratch: this many copies of the largest weight matrix

// FP32 GEMM with a long reduction (the weight gradients, K = the batch): the K range is cut
// into `split` slices, so that the few output tiles still give every SM work; each slice's
// partial tile goes to `scratch` and a second pass adds them in order (deterministic).
cudaError_t gemm_f32_splitk(const void* A, int M, const void* B, int N, int K, const EpiArgs& ep, float* scratch,
                            size_t scratch_floats, int num_sms, cudaStream_t s) {
  if (M % BM || K % BK || N % 64) return cudaErrorInvalidValue;
  const int BN = N % 128 == 0 ? 128 : 64;
  const int tiles = (N / BN) * (M / BM);
  int split = 1;
  for (int c = 2; c <= kMaxSplit; ++c)
    if ((K / BK) % c == 0 && tiles * c <= 2 * num_sms && (size_t)c * M * N <= scratch_floats) split = c;
  if (split == 1) return gemm<EPI_F32>(A, M, B, N, K, ep, s);
  EpiArgs ps = ep;
  ps.out_f32 = scratch;
  ps.ldo = N;
  ps.slice_stride = (size_t)M * N;
  cudaError_t e = BN == 128 ? gemm_launch<128, EPI_F32>(A, M, B, N, K, ps, s, split)
                            : gemm_launch<64, EPI_F32>(A, M, B, N, K, ps, s, split);
  if (e != cudaSuccess) return e;
  const size_t n = (size_t)M * N;
  splitk_reduce<<<(unsigned)std::min<size_t>((n + 255) / 256, 1216), 256, 0, s>>>(scratch, split, n, ep.out_f32);
  return cudaGetLastError();
}

inline size_t al(size_t x) { return (x + 255) / 256 * 256; }
}  // namespace

struct cf_mlp {
  int fin, kin, H, O, maxB, Bp_max;
  char* ws;
  // fp32 master parameters and Adam moments, contiguous: W1 b1 W2 b2 W3 b3
  float *w, *g, *m, *v;
  size_t nparam;
  size_t oW1, ob1, oW2, ob2, oW3, ob3;
  __nv_bfloat16 *W1b, *W2b, *W3b, *W2t, *W3t;
  __nv_bfloat16 *X0, *Z1, *H1, *Z2, *H2, *dY, *dA2, *dA1, *dYt, *H2t, *dA2t, *H1t, *dA1t, *X0t;
  float *Y, *loss, *part3, *part2, *part1, *splitk;
  size_t splitk_floats;
  int num_sms;
  int* err;
  long step;
};

static size_t mlp_layout(int fin, int H, int O, int maxB, cf_mlp* m) {
  int kin = (fin + 63) / 64 * 64;
  int Bp = (maxB + 127) / 128 * 128;
  size_t np = (size_t)H * kin + H + (size_t)H * H + H + (size_t)O * H + O;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off = al(off + bytes); return r; };
  size_t o_w = take(np * 4), o_g = take(np * 4), o_m = take(np * 4), o_v = take(np * 4);
  size_t o_W1b = take((size_t)H * kin * 2), o_W2b = take((size_t)H * H * 2), o_W3b = take((size_t)O * H * 2);
  size_t o_W2t = take((size_t)H * H * 2), o_W3t = take((size_t)O * H * 2);
  size_t o_X0 = take((size_t)Bp * kin * 2), o_Z1 = take((size_t)Bp * H * 2), o_H1 = take((size_t)Bp * H * 2);
  size_t o_Z2 = take((size_t)Bp * H * 2), o_H2 = take((size_t)Bp * H * 2), o_dY = take((size_t)Bp * O * 2);
  size_t o_dA2 = take((size_t)Bp * H * 2), o_dA1 = take((size_t)Bp * H * 2), o_dYt = take((size_t)Bp * O * 2);
  size_t o_H2t = take((size_t)Bp * H * 2), o_dA2t = take((size_t)Bp * H * 2), o_H1t = take((size_t)Bp * H * 2);
  size_t o_dA1t = take((size_t)Bp * H * 2), o_X0t = take((size_t)Bp * kin * 2);
  size_t o_Y = take((size_t)Bp * O * 4), o_loss = take(16), o_err = take(16);
  // the bias gradients' partial sums: dY per 64-row tile, dA2 and dA1 per 32-row chunk
  size_t o_part3 = take((size_t)(Bp / 64) * O * 4), o_part2 = take((size_t)(Bp / 32) * H * 4);
  size_t o_part1 = take((size_t)(Bp / 32) * H * 4);
  const size_t wmax = std::max((size_t)O * H, std::max((size_t)H * H, (size_t)H * kin));
  size_t o_splitk = take((size_t)kSplitScratch * wmax * 4);
  if (m) {
    char* b = m->ws;
    m->fin = fin; m->kin = kin; m->H = H; m->O = O; m->maxB = maxB; m->Bp_max = Bp;
    m->nparam = np;
    m->w = (float*)(b + o_w); m->g = (float*)(b + o_g); m->m = (float*)(b + o_m); m->v = (float*)(b + o_v);
    m->oW1 = 0; m->ob1 = m->oW1 + (size_t)H * kin; m->oW2 = m->ob1 + H; m->ob2 = m->oW2 + (size_t)H * H;
    m->oW3 = m->ob2 + H; m->ob3 = m->oW3 + (size_t)O * H;
    m->W1b = (__nv_bfloat16*)(b + o_W1b); m->W2b = (__nv_bfloat16*)(b + o_W2b); m->W3b = (__nv_bfloat16*)(b + o_W3b);
    m->W2t = (__nv_bfloat16*)(b + o_W2t); m->W3t = (__nv_bfloat16*)(b + o_W3t);
    m->X0 = (__nv_bfloat16*)(b + o_X0); m->Z1 = (__nv_bfloat16*)(b + o_Z1); m->H1 = (__nv_bfloat16*)(b + o_H1);
    m->Z2 = (__nv_bfloat16*)(b + o_Z2); m->H2 = (__nv_bfloat16*)(b + o_H2); m->dY = (__nv_bfloat16*)(b + o_dY);
    m->dA2 = (__nv_bfloat16*)(b + o_dA2); m->dA1 = (__nv_bfloat16*)(b + o_dA1); m->dYt = (__nv_bfloat16*)(b + o_dYt);
    m->H2t = (__nv_bfloat16*)(b + o_H2t); m->dA2t = (__nv_bfloat16*)(b + o_dA2t); m->H1t = (__nv_bfloat16*)(b + o_H1t);
    m->dA1t = (__nv_bfloat16*)(b + o_dA1t); m->X0t = (__nv_bfloat16*)(b + o_X0t);
    m->Y = (float*)(b + o_Y); m->loss = (float*)(b + o_loss); m->err = (int*)(b + o_err);
    m->part3 = (float*)(b + o_part3); m->part2 = (float*)(b + o_part2); m->part1 = (float*)(b + o_part1);
    m->splitk = (float*)(b + o_splitk);
    m->splitk_floats = (size_t)kSplitScratch * wmax;
  }
  return off;
}

static bool mlp_dims_ok(int fin, int H, int O) {
  return fin >= 1 && fin <= 256 && H >= 64 && H <= 1024 && H % 128 == 0 && O >= 128 && O <= 4096 && O % 256 == 0;
}

extern "C" cf_status cf_mlp_workspace_bytes(int32_t fin, int32_t hidden, int32_t fout, int32_t max_batch, size_t* bytes) {
  if (!bytes || !mlp_dims_ok(fin, hidden, fout) || max_batch < 1 || max_batch > (1 << 20))
    return mfail(CF_ERR_INVALID_ARGUMENT, "mlp dims: 1 <= in <= 256, hidden % 128 == 0, out % 256 == 0");
  *bytes = mlp_layout(fin, hidden, fout, max_batch, nullptr);
  return CF_OK;
}

static void upd_bf16(cf_mlp* m, cudaStream_t s) {
  auto go = [&](size_t off, int rows, int cols, __nv_bfloat16* wb, __nv_bfloat16* wt) {
    int n = rows * cols;
    to_bf16<<<(n + 255) / 256, 256, 0, s>>>(m->w + off, n, wb, wt, rows, cols);
  };
  go(m->oW1, m->H, m->kin, m->W1b, nullptr);
  go(m->oW2, m->H, m->H, m->W2b, m->W2t);
  go(m->oW3, m->O, m->H, m->W3b, m->W3t);
}

extern "C" cf_status cf_mlp_create(int32_t fin, int32_t hidden, int32_t fout, int32_t max_batch, const float* params,
                                   void* device_workspace, size_t bytes, void* stream, cf_mlp** out) {
  size_t need = 0;
  cf_status st = cf_mlp_workspace_bytes(fin, hidden, fout, max_batch, &need);
  if (st != CF_OK) return st;
  if (!out || !device_workspace || bytes < need || (reinterpret_cast<uintptr_t>(device_workspace) & 255))
    return mfail(CF_ERR_INVALID_ARGUMENT, "mlp workspace missing, too small or not 256-byte aligned");
  if (!params) return mfail(CF_ERR_INVALID_ARGUMENT, "initial parameters required");
  if (!get_encoder()) return mfail(CF_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  cf_mlp* m = new (std::nothrow) cf_mlp();
  if (!m) return mfail(CF_ERR_OUT_OF_MEMORY, "mlp allocation");
  m->ws = static_cast<char*>(device_workspace);
  mlp_layout(fin, hidden, fout, max_batch, m);
  {
    int dev = 0;
    m->num_sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, dev);
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(m->ws, 0, need, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->w, params, m->nparam * 4, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) {
    upd_bf16(m, s);
    e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) {
    delete m;
    return mfail(CF_ERR_CUDA, cudaGetErrorString(e));
  }
  m->step = 0;
  *out = m;
  return CF_OK;
}

extern "C" void cf_mlp_destroy(cf_mlp* m) { delete m; }

extern "C" cf_status cf_mlp_param_count(const cf_mlp* m, int64_t* n) {
  if (!m || !n) return mfail(CF_ERR_INVALID_ARGUMENT, "null argument");
  *n = (int64_t)m->nparam;
  return CF_OK;
}

// train: the hidden layers' GEMMs also write H1^T and H2^T [H x Bp], the K-major operands of
// the weight gradients
static cf_status forward(cf_mlp* m, const float* x, int B, cudaStream_t s, bool train = false) {
  const int Bp = (B + 127) / 128 * 128;
  int n = Bp * m->kin;
  pack_input<<<(n + 255) / 256, 256, 0, s>>>(x, B, m->fin, Bp, m->kin, m->X0);
  EpiArgs e1{};
  e1.bias = m->w + m->ob1; e1.out_bf16 = m->H1; e1.out_z = m->Z1; e1.ldo = m->H; e1.m_valid = Bp; e1.err = m->err;
  if (train) { e1.out_t = m->H1t; e1.ldt = Bp; }
  cudaError_t e = gemm<EPI_BIAS_GELU>(m->X0, Bp, m->W1b, m->H, m->kin, e1, s);
  EpiArgs e2 = e1;
  e2.bias = m->w + m->ob2; e2.out_bf16 = m->H2; e2.out_z = m->Z2;
  if (train) e2.out_t = m->H2t;
  if (e == cudaSuccess) e = gemm<EPI_BIAS_GELU>(m->H1, Bp, m->W2b, m->H, m->H, e2, s);
  EpiArgs e3{};
  e3.bias = m->w + m->ob3; e3.out_f32 = m->Y; e3.ldo = m->O; e3.m_valid = Bp; e3.err = m->err;
  if (e == cudaSuccess) e = gemm<EPI_BIAS_F32>(m->H2, Bp, m->W3b, m->O, m->H, e3, s);
  if (e != cudaSuccess) return mfail(CF_ERR_CUDA, cudaGetErrorString(e));
  return CF_OK;
}

extern "C" cf_status cf_mlp_forward(cf_mlp* m, const float* x, int32_t B, float* y, void* stream) {
  if (!m || !x || !y || B < 1 || B > m->maxB) return mfail(CF_ERR_INVALID_ARGUMENT, "bad mlp forward arguments");
  cudaStream_t s = (cudaStream_t)stream;
  cf_status st = forward(m, x, B, s);
  if (st != CF_OK) return st;
  if (cudaMemcpyAsync(y, m->Y, (size_t)B * m->O * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return mfail(CF_ERR_CUDA, "copy out");
  return CF_OK;
}

// gradients of the Gaussian NLL into m->g (fp32, parameter layout); loss into m->loss
static cf_status backward(cf_mlp* m, const float* target, int B, float lo, float hi, cudaStream_t s) {
  const int Bp = (B + 127) / 128 * 128, H = m->H, O = m->O, D = O / 2;
  cudaMemsetAsync(m->loss, 0, 4, s);
  nll_grad<<<dim3(D / 64, Bp / 64), dim3(32, 8), 0, s>>>(m->Y, target, B, Bp, D, lo, hi, m->dY, m->dYt, m->loss,
                                                         m->part3);
  auto colsum = [&](const float* part, int N, int slices, float* db) {
    bias_grad_final<<<N / 64, 256, 0, s>>>(part, N, slices, db);
  };
  dim3 tb(32, 8);
  auto T = [&](const __nv_bfloat16* in, int R, int C, __nv_bfloat16* out) {
    transpose_bf16<<<dim3((C + 63) / 64, (R + 63) / 64), tb, 0, s>>>(in, R, C, out);
  };
  cudaError_t e = cudaSuccess;
  // layer 3: dW3 = dY^T H2, db3 = colsum dY, dH2 = dY W3 (times gelu'(Z2)); dY^T comes from
  // nll_grad and H2^T from the forward pass, dA2^T and dA1^T from the GELU-derivative epilogues
  EpiArgs ew{};
  ew.out_f32 = m->g + m->oW3; ew.ldo = H; ew.m_valid = O; ew.err = m->err;
  e = gemm_f32_splitk(m->dYt, O, m->H2t, H, Bp, ew, m->splitk, m->splitk_floats, m->num_sms, s);
  colsum(m->part3, O, Bp / 64, m->g + m->ob3);
  EpiArgs eb{};
  eb.out_bf16 = m->dA2; eb.z = m->Z2; eb.ldo = H; eb.m_valid = Bp; eb.err = m->err;
  eb.out_t = m->dA2t; eb.ldt = Bp; eb.colsum = m->part2;
  if (e == cudaSuccess) e = gemm<EPI_GELU_BWD>(m->dY, Bp, m->W3t, H, O, eb, s);
  // layer 2
  ew.out_f32 = m->g + m->oW2; ew.ldo = H; ew.m_valid = H;
  if (e == cudaSuccess) e = gemm_f32_splitk(m->dA2t, H, m->H1t, H, Bp, ew, m->splitk, m->splitk_floats, m->num_sms, s);
  colsum(m->part2, H, Bp / 128, m->g + m->ob2);
  eb.out_bf16 = m->dA1; eb.z = m->Z1; eb.out_t = m->dA1t; eb.colsum = m->part1;
  if (e == cudaSuccess) e = gemm<EPI_GELU_BWD>(m->dA2, Bp, m->W2t, H, H, eb, s);
  // layer 1
  T(m->X0, Bp, m->kin, m->X0t);
  ew.out_f32 = m->g + m->oW1; ew.ldo = m->kin; ew.m_valid = H;
  if (e == cudaSuccess) e = gemm_f32_splitk(m->dA1t, H, m->X0t, m->kin, Bp, ew, m->splitk, m->splitk_floats, m->num_sms, s);
  colsum(m->part1, H, Bp / 128, m->g + m->ob1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return mfail(CF_ERR_CUDA, cudaGetErrorString(e));
  return CF_OK;
}

extern "C" cf_status cf_mlp_gradients(cf_mlp* m, const float* x, const float* target, int32_t B, float logstd_lo,
                                      float logstd_hi, float* grads, float* loss, void* stream) {
  if (!m || !x || !target || B < 1 || B > m->maxB) return mfail(CF_ERR_INVALID_ARGUMENT, "bad mlp arguments");
  cudaStream_t s = (cudaStream_t)stream;
  cf_status st = forward(m, x, B, s, true);
  if (st == CF_OK) st = backward(m, target, B, logstd_lo, logstd_hi, s);
  if (st != CF_OK) return st;
  if (grads) cudaMemcpyAsync(grads, m->g, m->nparam * 4, cudaMemcpyDeviceToDevice, s);
  if (loss) cudaMemcpyAsync(loss, m->loss, 4, cudaMemcpyDeviceToDevice, s);
  return CF_OK;
}

extern "C" cf_status cf_mlp_train_step(cf_mlp* m, const float* x, const float* target, int32_t B, float lr,
                                       float logstd_lo, float logstd_hi, float* loss, void* stream) {
  cf_status st = cf_mlp_gradients(m, x, target, B, logstd_lo, logstd_hi, nullptr, loss, stream);
  if (st != CF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  m->step += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
  auto go = [&](size_t off, int rows, int cols, __nv_bfloat16* wb, __nv_bfloat16* wt) {
    int n = rows * cols;
    adam<<<(n + 255) / 256, 256, 0, s>>>(m->w + off, m->g + off, m->m + off, m->v + off, n, lr, b1, b2, eps, c1, c2, wb,
                                         wt, rows, cols);
  };
  go(m->oW1, m->H, m->kin, m->W1b, nullptr);
  go(m->ob1, 1, m->H, nullptr, nullptr);
  go(m->oW2, m->H, m->H, m->W2b, m->W2t);
  go(m->ob2, 1, m->H, nullptr, nullptr);
  go(m->oW3, m->O, m->H, m->W3b, m->W3t);
  go(m->ob3, 1, m->O, nullptr, nullptr);
  if (cudaGetLastError() != cudaSuccess) return mfail(CF_ERR_CUDA, "adam launch");
  return CF_OK;
}

extern "C" cf_status cf_mlp_get_params(const cf_mlp* m, float* params, void* stream) {
  if (!m || !params) return mfail(CF_ERR_INVALID_ARGUMENT, "null argument");
  if (cudaMemcpyAsync(params, m->w, m->nparam * 4, cudaMemcpyDeviceToDevice, (cudaStream_t)stream) != cudaSuccess)
    return mfail(CF_ERR_CUDA, "copy params");
  return CF_OK;
}

extern "C" cf_status cf_mlp_status(cf_mlp* m, void* stream) {
  if (!m) return mfail(CF_ERR_INVALID_ARGUMENT, "null argument");
  int w = 0;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&w, m->err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return mfail(CF_ERR_CUDA, "read mlp status");
  if (w & CF_FLAG_TIMEOUT) return mfail(CF_ERR_TIMEOUT, "a tensor-core pipeline wait gave up");
  return CF_OK;
}
