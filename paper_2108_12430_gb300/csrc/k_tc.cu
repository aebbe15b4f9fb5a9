// Tensor-core (tcgen05) implicit-GEMM convolution for sm_103a.
//
// Every Conv1d / ConvTranspose1d layer of the two networks runs here as
//   D[m][n] = sum_steps A_step[m][16 k] * B_step[n][16 k]
// with M = 128 output positions per MMA (one TMEM lane each), N = output
// channels (padded to a multiple of 16) and K-steps of 16 BF16 (or 32 e4m3)
// inputs.  A K-step is made of two 16-byte "slices": 8 (16) input channels of
// one tap, read from an input phase plane at a row shift.  Because the input
// tile sits in shared memory in the no-swizzle K-major core-matrix layout
// (16-byte rows, 8-row core matrices), a tap is only a different descriptor
// start address: the im2col matrix is never formed.
//   conv, stride s:  output t, tap k reads input s t + k - p = phase
//                    (k - p) mod s, row t + floor((k - p) / s);
//   convT, stride 2: output u = 2 m + psi gathers taps k with psi + p - k
//                    even from input row m + (psi + p - k) / 2 (two output
//                    phases = two accumulator chains).
// The BatchNorm is folded into the weights (FP64, host); bias, activation
// and an optional residual are applied in the epilogue from TMEM.
//
// Data movement: the input tile (all channel groups and phases, plus the tap
// halo) arrives by one bulk TMA copy per plane; the weight image streams
// through a ring of stages by bulk TMA; one thread issues the MMAs; all four
// warps drain TMEM with tcgen05.ld.  Every wait is bounded (1 s) and reports
// through an error flag instead of hanging.
#include <cuda_fp8.h>
#include <string.h>

#include <algorithm>

#include "gw_internal.h"

namespace gw {

namespace {

constexpr int kThreads = 128;
constexpr uint64_t kWaitNs = 1000000000ull;  // bounded waits: 1 s
constexpr int kErrWaitA = 1, kErrWaitB = 2, kErrWaitEmpty = 4, kErrWaitDone = 8;

struct TcParams {
  const char* in;
  int64_t in_off0, in_b, in_boff, in_g, in_p;  // bytes (boff in 16-byte rows)
  int in_P, in_L, G;
  int MT, rows, dmin, n_chains, chainP, mout0, mout1, lout;
  const char* wimg;
  const uint32_t* table;
  int n_steps, npad, sps, nst, step_bytes, a_bytes, ncols;
  uint32_t idesc;
  int fp8;
  const float* bias;
  const float* wscale;  // FP8: per output channel dequantisation scale
  int cout, act;
  char* out;
  int64_t out_b, out_g, out_p;  // bytes
  int out_P, fp32_single, fp8_out;
  float out_scale;
  const char* res;
  int64_t res_b, res_g, res_p;  // bytes
  int res_P, res_fp8;
  float res_scale;
  int* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits for the barrier phase with a time limit; on timeout records `code`.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer() - t0 > kWaitNs) {
      atomicOr(err, code);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void st_shared_zero16(uint32_t addr) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(addr), "r"(0) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// Shared-memory matrix descriptor, no swizzle, K-major: start address, LBO =
// byte distance between the two K-adjacent core matrices, SBO = byte distance
// between core matrices adjacent in M/N; bits 46-48 hold the fixed 0b001.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_f8(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float act_fn(float v, int act) {
  if (act == ACT_TANH) return tanhf(v);
  if (act == ACT_RELU) return fmaxf(v, 0.f);
  return v;
}

// Byte offset (for M sub-tile 0) of the 16-byte slice coded as g | phi << 8 | dd << 10.
__device__ __forceinline__ uint32_t slice_off(uint32_t code, int P, int rows) {
  const uint32_t g = code & 0xFFu, phi = (code >> 8) & 3u, dd = (code >> 10) & 63u;
  return ((g * (uint32_t)P + phi) * (uint32_t)rows + dd) * 16u;
}

__global__ void __launch_bounds__(kThreads, 1) conv_tc_kernel(const TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  const uint32_t sA = smem_u32(smem);
  const uint32_t sB = sA + (uint32_t)p.a_bytes;
  const uint32_t stage_bytes = (uint32_t)(p.sps * p.step_bytes);
  uint64_t* bars = (uint64_t*)(smem + p.a_bytes + p.nst * stage_bytes);
  uint32_t* tslot = (uint32_t*)(bars + 2 + 2 * p.nst);
  volatile uint32_t* abort_flag = tslot + 1;
  uint32_t* s_table = tslot + 2;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t barA = smem_u32(&bars[0]);
  const uint32_t barD = smem_u32(&bars[1 + 2 * p.nst]);
  const int m0 = blockIdx.x * 128 * p.MT;
  const int b = blockIdx.y;

  if (tid == 0) {
    mbar_init(barA, 1);
    for (int i = 0; i < p.nst; ++i) {
      mbar_init(smem_u32(&bars[1 + i]), 1);
      mbar_init(smem_u32(&bars[1 + p.nst + i]), 1);
    }
    mbar_init(barD, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  for (int i = tid; i < 2 * p.n_steps; i += kThreads) s_table[i] = p.table[i];
  if (warp == 0) tmem_alloc(smem_u32(tslot), (uint32_t)p.ncols);

  // Rows of the input tile outside the layer's input are its zero padding.
  const int planes = p.G * p.in_P;
  for (int plane = 0; plane < planes; ++plane) {
    const int phi = plane % p.in_P;
    const int Lp = (p.in_L - phi + p.in_P - 1) / p.in_P;
    const int r0 = max(0, -m0 - p.dmin);
    const int r1 = max(r0, min(p.rows, Lp - m0 - p.dmin));
    for (int r = tid; r < p.rows; r += kThreads)
      if (r < r0 || r >= r1) st_shared_zero16(sA + (uint32_t)(plane * p.rows + r) * 16u);
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (tid == 0) {
    // input tile: one bulk copy per (channel group, phase) plane
    uint32_t total = 0;
    for (int plane = 0; plane < planes; ++plane) {
      const int phi = plane % p.in_P;
      const int Lp = (p.in_L - phi + p.in_P - 1) / p.in_P;
      const int r0 = max(0, -m0 - p.dmin);
      const int r1 = max(r0, min(p.rows, Lp - m0 - p.dmin));
      total += (uint32_t)(r1 - r0) * 16u;
    }
    if (total) {
      mbar_expect_tx(barA, total);
      for (int plane = 0; plane < planes; ++plane) {
        const int g = plane / p.in_P, phi = plane % p.in_P;
        const int Lp = (p.in_L - phi + p.in_P - 1) / p.in_P;
        const int r0 = max(0, -m0 - p.dmin);
        const int r1 = max(r0, min(p.rows, Lp - m0 - p.dmin));
        if (r1 <= r0) continue;
        const char* src = p.in + p.in_off0 + (int64_t)b * p.in_b + (int64_t)g * p.in_g + (int64_t)phi * p.in_p +
                          ((int64_t)(m0 + p.dmin + r0) + (int64_t)b * p.in_boff) * 16;
        bulk_g2s(sA + (uint32_t)(plane * p.rows + r0) * 16u, src, (uint32_t)(r1 - r0) * 16u, barA);
      }
    } else {
      mbar_arrive(barA);
    }
  }

  const int n_chunks = (p.n_steps + p.sps - 1) / p.sps;
  if (tid == 32) {
    // weight producer: chunks of sps K-steps through nst stages
    for (int c = 0; c < n_chunks; ++c) {
      const int st = c % p.nst;
      if (c >= p.nst &&
          !mbar_wait(smem_u32(&bars[1 + p.nst + st]), (uint32_t)((c / p.nst) - 1) & 1u, p.err, kErrWaitEmpty))
        break;
      const int s0 = c * p.sps, s1 = min(p.n_steps, s0 + p.sps);
      const uint32_t bytes = (uint32_t)((s1 - s0) * p.step_bytes);
      const uint32_t full = smem_u32(&bars[1 + st]);
      mbar_expect_tx(full, bytes);
      bulk_g2s(sB + (uint32_t)st * stage_bytes, p.wimg + (int64_t)s0 * p.step_bytes, bytes, full);
    }
  }

  if (tid == 0) {
    // single-thread MMA issue
    bool ok = mbar_wait(barA, 0, p.err, kErrWaitA);
    tc_fence_after();
    const uint32_t sbo = 128u, b_lbo = (uint32_t)p.npad * 16u;
    for (int c = 0; ok && c < n_chunks; ++c) {
      const int st = c % p.nst;
      if (!mbar_wait(smem_u32(&bars[1 + st]), (uint32_t)(c / p.nst) & 1u, p.err, kErrWaitB)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const int s0 = c * p.sps, s1 = min(p.n_steps, s0 + p.sps);
      for (int s = s0; s < s1; ++s) {
        const uint32_t w0 = s_table[2 * s], w1 = s_table[2 * s + 1];
        const uint32_t chain = w1 & 15u, acc = ((w1 >> 4) & 1u) ? 0u : 1u;
        const uint32_t o0 = slice_off(w0 & 0xFFFFu, p.in_P, p.rows);
        const uint32_t o1 = slice_off(w0 >> 16, p.in_P, p.rows);
        const uint64_t bdesc = make_desc(sB + (uint32_t)st * stage_bytes + (uint32_t)(s - s0) * p.step_bytes, b_lbo, sbo);
        for (int mt = 0; mt < p.MT; ++mt) {
          const uint64_t adesc = make_desc(sA + o0 + (uint32_t)mt * 2048u, o1 - o0, sbo);
          const uint32_t d = tmem + (chain * (uint32_t)p.MT + (uint32_t)mt) * (uint32_t)p.npad;
          if (p.fp8)
            mma_f8(d, adesc, bdesc, p.idesc, acc);
          else
            mma_f16(d, adesc, bdesc, p.idesc, acc);
        }
      }
      mma_commit(smem_u32(&bars[1 + p.nst + st]));
    }
    if (!ok) *abort_flag = 1u;
    mma_commit(barD);
  }
  __syncthreads();

  // epilogue: TMEM -> registers -> bias / residual / activation -> global
  const bool done = mbar_wait(barD, 0, p.err, kErrWaitDone);
  __syncwarp();
  tc_fence_after();
  if (done && *abort_flag == 0u) {
    const int row = warp * 32 + lane;
    for (int c = 0; c < p.n_chains; ++c) {
      const int mout = c ? p.mout1 : p.mout0;
      for (int mt = 0; mt < p.MT; ++mt) {
        const int m = m0 + mt * 128 + row;
        const bool valid = m < mout;
        const int u = p.chainP * m + c;
        for (int j = 0; j < p.npad / 16; ++j) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((c * p.MT + mt) * p.npad + j * 16), v);
          if (!valid) continue;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int n0 = j * 16 + h * 8;
            if (n0 >= p.cout) continue;
            float x[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int n = n0 + i;
              float a = v[h * 8 + i];
              if (n < p.cout) {
                if (p.wscale) a *= p.wscale[n];
                a += p.bias[n];
              } else {
                a = 0.f;
              }
              x[i] = a;
            }
            if (p.res) {
              if (p.res_fp8) {
                const int go = n0 / 16;
                const char* rp = p.res + (int64_t)b * p.res_b + (int64_t)go * p.res_g + (int64_t)(u % p.res_P) * p.res_p +
                                 (int64_t)(u / p.res_P) * 16 + (n0 % 16);
                const uint2 rv = *reinterpret_cast<const uint2*>(rp);
                const __nv_fp8_e4m3* r8 = reinterpret_cast<const __nv_fp8_e4m3*>(&rv);
#pragma unroll
                for (int i = 0; i < 8; ++i) x[i] += float(r8[i]) * p.res_scale;
              } else {
                const int go = n0 / 8;
                const char* rp = p.res + (int64_t)b * p.res_b + (int64_t)go * p.res_g + (int64_t)(u % p.res_P) * p.res_p +
                                 (int64_t)(u / p.res_P) * 16;
                const uint4 rv = *reinterpret_cast<const uint4*>(rp);
                const __nv_bfloat16* r16 = reinterpret_cast<const __nv_bfloat16*>(&rv);
#pragma unroll
                for (int i = 0; i < 8; ++i) x[i] += __bfloat162float(r16[i]);
              }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = act_fn(x[i], p.act);
            if (p.fp32_single) {
              if (n0 == 0) reinterpret_cast<float*>(p.out + (int64_t)b * p.out_b)[u] = x[0];
            } else if (p.fp8_out) {
              const int go = n0 / 16;
              __align__(8) __nv_fp8_e4m3 o8[8];
#pragma unroll
              for (int i = 0; i < 8; ++i) o8[i] = __nv_fp8_e4m3(x[i] * p.out_scale);
              char* op = p.out + (int64_t)b * p.out_b + (int64_t)go * p.out_g + (int64_t)(u % p.out_P) * p.out_p +
                         (int64_t)(u / p.out_P) * 16 + (n0 % 16);
              *reinterpret_cast<uint2*>(op) = *reinterpret_cast<const uint2*>(o8);
            } else {
              const int go = n0 / 8;
              __align__(16) __nv_bfloat16 o16[8];
#pragma unroll
              for (int i = 0; i < 8; ++i) o16[i] = __float2bfloat16_rn(x[i]);
              char* op = p.out + (int64_t)b * p.out_b + (int64_t)go * p.out_g + (int64_t)(u % p.out_P) * p.out_p +
                         (int64_t)(u / p.out_P) * 16;
              *reinterpret_cast<uint4*>(op) = *reinterpret_cast<const uint4*>(o16);
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, (uint32_t)p.ncols);
}

// FP32 [B][C][*] -> blocked layout (bf16 rows of 8 channels, or e4m3 rows of 16).
__global__ void to_blocked_kernel(const float* __restrict__ x, int64_t xb, int64_t xc, int B, int C, int L,
                                  const float* __restrict__ mean, const float* __restrict__ istd, float scale,
                                  char* __restrict__ out, int64_t ob, int64_t og, int64_t op, int P, int fp8) {
  const int cg = fp8 ? 16 : 8;
  const int G = (C + cg - 1) / cg;
  const int64_t total = (int64_t)B * G * L;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(e % L);
    const int g = (int)((e / L) % G);
    const int b = (int)(e / ((int64_t)L * G));
    float v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int c = g * cg + i;
      float a = 0.f;
      if (i < cg && c < C) {
        a = x[(int64_t)b * xb + (int64_t)c * xc + t];
        if (mean) a = (a - mean[c]) * istd[c];
      }
      v[i] = a;
    }
    char* dst = out + (int64_t)b * ob + (int64_t)g * og + (int64_t)(t % P) * op + (int64_t)(t / P) * 16;
    if (fp8) {
      __align__(16) __nv_fp8_e4m3 o8[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) o8[i] = __nv_fp8_e4m3(v[i] * scale);
      *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(o8);
    } else {
      __align__(16) __nv_bfloat16 o16[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) o16[i] = __float2bfloat16_rn(v[i]);
      *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(o16);
    }
  }
}

// Global average pool of a blocked activation + linear head; one CTA per item.
__global__ void gap_linear_blocked_kernel(const char* __restrict__ in, int64_t ib, int64_t ig, int64_t ip, int P,
                                          int L, int C, int fp8, float in_scale, const float* __restrict__ w,
                                          const float* __restrict__ bias, float* __restrict__ out) {
  __shared__ float red[8];
  const int b = blockIdx.x;
  const int cg = fp8 ? 16 : 8;
  float part = 0.f;
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    const int g = c / cg, i = c % cg;
    float s = 0.f;
    for (int t = 0; t < L; ++t) {
      const char* row = in + (int64_t)b * ib + (int64_t)g * ig + (int64_t)(t % P) * ip + (int64_t)(t / P) * 16;
      s += fp8 ? float(reinterpret_cast<const __nv_fp8_e4m3*>(row)[i]) * in_scale
               : __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(row)[i]);
    }
    part = fmaf(s / (float)L, w[c], part);
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) v += red[i];
    out[b] = v + bias[0];
  }
}

inline int pmod_i(int a, int m) { return ((a % m) + m) % m; }

}  // namespace

int tc_supported() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3;
}

// Lowers one folded layer to K-steps of two 16-byte slices and packs the B
// operand image: per step [2 K-halves][npad rows][16 bytes], K-major core
// matrices with LBO = npad * 16 bytes and SBO = 128 bytes.
// Host only; fills L's lowering fields and returns the image, table and (FP8)
// per-channel weight scales.
static void lower_layer(LayerDev& L, const std::vector<double>& wf, bool fp8, std::vector<uint8_t>& img,
                        std::vector<uint32_t>& table, std::vector<float>& wscale) {
  const LayerSpec& s = L.s;
  const int cg = fp8 ? 16 : 8;
  const int G = (s.cin + cg - 1) / cg;
  const int pin = s.transposed ? 1 : s.stride;
  int npad = std::max(16, (s.cout + 15) / 16 * 16);
  GW_CHECK_ARG(npad <= 256, "C_out above 256 is not supported by the tensor-core path");
  GW_CHECK_ARG(G <= 255, "too many input channels");
  struct Tap { int k, phi, d; };
  std::vector<std::vector<Tap>> chains;
  if (!s.transposed) {
    std::vector<Tap> ch;
    for (int k = 0; k < s.k; ++k) {
      const int phi = pmod_i(k - s.pad_l, pin);
      ch.push_back({k, phi, (k - s.pad_l - phi) / pin});
    }
    chains.push_back(ch);
  } else {
    GW_CHECK_ARG(s.stride == 2 && s.pad_l == s.pad_r, "transposed conv must have stride 2 and symmetric padding");
    for (int psi = 0; psi < 2; ++psi) {
      std::vector<Tap> ch;
      for (int k = 0; k < s.k; ++k)
        if (pmod_i(psi + s.pad_l - k, 2) == 0) ch.push_back({k, 0, (psi + s.pad_l - k) / 2});
      chains.push_back(ch);
    }
  }
  int dmin = 1 << 30, dmax = -(1 << 30);
  for (auto& ch : chains)
    for (auto& t : ch) {
      dmin = std::min(dmin, t.d);
      dmax = std::max(dmax, t.d);
    }
  GW_CHECK_ARG(dmax - dmin < 64, "tap span too large");
  struct Slice { int g, phi, dd, k; bool dummy; };
  auto key = [](const Slice& a) { return (a.g * 4 + a.phi) * 64 + a.dd; };
  struct Step { Slice a, b; int chain; bool first; };
  std::vector<Step> steps;
  for (size_t ci = 0; ci < chains.size(); ++ci) {
    std::vector<std::pair<Slice, Slice>> st;
    std::vector<Slice> left;
    for (auto& t : chains[ci]) {
      int g = 0;
      for (; g + 1 < G; g += 2)
        st.push_back({{g, t.phi, t.d - dmin, t.k, false}, {g + 1, t.phi, t.d - dmin, t.k, false}});
      if (g < G) left.push_back({g, t.phi, t.d - dmin, t.k, false});
    }
    std::sort(left.begin(), left.end(), [&](const Slice& a, const Slice& b) { return key(a) < key(b); });
    for (size_t i = 0; i < left.size(); i += 2) {
      if (i + 1 < left.size()) {
        st.push_back({left[i], left[i + 1]});
      } else {
        Slice d = left[i];
        d.dummy = true;
        st.push_back({left[i], d});
      }
    }
    for (size_t i = 0; i < st.size(); ++i) {
      Slice a = st[i].first, b = st[i].second;
      if (key(b) < key(a)) std::swap(a, b);
      steps.push_back({a, b, (int)ci, i == 0});
    }
  }
  GW_CHECK_ARG(steps.size() <= 4096, "too many K-steps");
  const int n_steps = (int)steps.size();
  const size_t step_bytes = 32 * (size_t)npad;
  img.assign(n_steps * step_bytes, 0);
  table.assign(2 * n_steps, 0u);
  // FP8: per-output-channel weight scale so that max |w| maps to 448
  wscale.assign(s.cout, 1.f);
  if (fp8) {
    for (int o = 0; o < s.cout; ++o) {
      double mx = 0;
      for (size_t e = 0; e < (size_t)s.cin * s.k; ++e) mx = std::max(mx, std::fabs(wf[(size_t)o * s.cin * s.k + e]));
      wscale[o] = mx > 0 ? (float)(mx / 448.0) : 1.f;
    }
  }
  for (int si = 0; si < n_steps; ++si) {
    const Step& st = steps[si];
    for (int half = 0; half < 2; ++half) {
      const Slice& sl = half ? st.b : st.a;
      for (int n = 0; n < npad; ++n)
        for (int kk = 0; kk < cg; ++kk) {
          const int c = sl.g * cg + kk;
          double v = 0.0;
          if (!sl.dummy && n < s.cout && c < s.cin) v = wf[((size_t)n * s.cin + c) * s.k + sl.k];
          uint8_t* dst = img.data() + si * step_bytes + ((size_t)half * npad + n) * 16;
          if (fp8) {
            __nv_fp8_e4m3 q((float)(v / wscale[n < s.cout ? n : 0]));
            memcpy(dst + kk, &q, 1);
          } else {
            __nv_bfloat16 q = __float2bfloat16_rn((float)v);
            memcpy(dst + kk * 2, &q, 2);
          }
        }
    }
    auto code = [](const Slice& a) { return (uint32_t)a.g | ((uint32_t)a.phi << 8) | ((uint32_t)a.dd << 10); };
    table[2 * si] = code(st.a) | (code(st.b) << 16);
    table[2 * si + 1] = (uint32_t)st.chain | ((st.first ? 1u : 0u) << 4);
  }
  L.n_steps = n_steps;
  L.npad = npad;
  L.gin = G;
  L.pin = pin;
  L.n_chains = (int)chains.size();
  L.dspan = dmax - dmin;
  L.dmin = dmin;
}

void tc_pack_layer(LayerDev& L, const std::vector<double>& wf, int precision, gw_ctx* ctx, size_t* counter,
                   std::vector<void*>& allocs) {
  const LayerSpec& s = L.s;
  const bool fp8 = precision == GW_FP8;
  std::vector<uint8_t> img;
  std::vector<uint32_t> table;
  std::vector<float> wscale;
  lower_layer(L, wf, fp8, img, table, wscale);
  void* d_img = dev_alloc(ctx, img.size(), counter);
  allocs.push_back(d_img);
  GW_CUDA(cudaMemcpy(d_img, img.data(), img.size(), cudaMemcpyHostToDevice));
  uint32_t* d_tab = (uint32_t*)dev_alloc(ctx, table.size() * 4, counter);
  allocs.push_back(d_tab);
  GW_CUDA(cudaMemcpy(d_tab, table.data(), table.size() * 4, cudaMemcpyHostToDevice));
  if (fp8) {
    // dequantisation per output channel: weight scale / scale of the input activations
    std::vector<float> deq(s.cout);
    for (int o = 0; o < s.cout; ++o) deq[o] = wscale[o] / L.act_scale;
    float* d_sc = (float*)dev_alloc(ctx, deq.size() * 4, counter);
    allocs.push_back(d_sc);
    GW_CUDA(cudaMemcpy(d_sc, deq.data(), deq.size() * 4, cudaMemcpyHostToDevice));
    L.wscale = d_sc;
  }
  L.wq = d_img;
  L.table = d_tab;
}

// Host-side launch plan (tile size, staging, TMEM columns, descriptors' idesc).
static void plan_conv_tc(TcParams& q, const LayerDev& L, bool fp8, const TcIn& in, int lout, const TcOut& out,
                         int* err, size_t* smem_out, dim3* grid_out, int B) {
  const LayerSpec& s = L.s;
  const int esz = fp8 ? 1 : 2;
  GW_CHECK_ARG(in.P == L.pin, "input phase count does not match the layer");
  q = TcParams{};
  q.in = (const char*)in.p;
  q.in_off0 = in.off0 * esz;
  q.in_b = in.bstride * esz;
  q.in_boff = in.boff;
  q.in_g = in.gstride * esz;
  q.in_p = in.pstride * esz;
  q.in_P = in.P;
  q.in_L = in.L;
  q.G = L.gin;
  q.n_chains = L.n_chains;
  q.chainP = s.transposed ? 2 : 1;
  q.mout0 = (lout + q.chainP - 1) / q.chainP;
  q.mout1 = s.transposed ? lout / 2 : 0;
  q.lout = lout;
  q.dmin = L.dmin;
  const int cols_per_mt = L.n_chains * L.npad;
  int MT = std::max(1, std::min(8, 128 / cols_per_mt));
  const int tiles_needed = (q.mout0 + 127) / 128;
  MT = std::min(MT, std::max(1, tiles_needed));
  auto a_bytes_for = [&](int mt) { return (size_t)L.gin * L.pin * (128 * mt + L.dspan) * 16; };
  while (MT > 1 && a_bytes_for(MT) > 96 * 1024) --MT;
  q.MT = MT;
  q.rows = 128 * MT + L.dspan;
  q.a_bytes = (int)((a_bytes_for(MT) + 127) / 128 * 128);
  q.step_bytes = 32 * L.npad;
  const size_t wbytes = (size_t)L.n_steps * q.step_bytes;
  const size_t budget = 200 * 1024;
  if (q.a_bytes + wbytes <= budget - 4096) {
    q.sps = L.n_steps;
    q.nst = 1;
  } else {
    q.sps = std::max(1, 32768 / q.step_bytes);
    const int n_chunks = (L.n_steps + q.sps - 1) / q.sps;
    q.nst = std::min(4, n_chunks);
    while (q.nst > 1 && q.a_bytes + (size_t)q.nst * q.sps * q.step_bytes > budget - 4096) --q.nst;
  }
  q.wimg = (const char*)L.wq;
  q.table = L.table;
  q.n_steps = L.n_steps;
  q.npad = L.npad;
  int ncols = 32;
  while (ncols < cols_per_mt * MT) ncols *= 2;
  GW_CHECK_ARG(ncols <= 512, "accumulators exceed tensor memory");
  q.ncols = ncols;
  // instruction descriptor: D = F32, A/B = BF16 (kind::f16) or E4M3 (kind::f8f6f4),
  // both K-major, N >> 3 at bit 17, M >> 4 at bit 24
  q.idesc = (1u << 4) | (fp8 ? 0u : ((1u << 7) | (1u << 10))) | ((uint32_t)(L.npad >> 3) << 17) |
            ((uint32_t)(128 >> 4) << 24);
  q.fp8 = fp8;
  q.bias = L.b;
  q.wscale = L.wscale;
  q.cout = s.cout;
  q.act = s.act;
  q.out = (char*)out.p;
  const int oesz = out.fp32_single ? 4 : (out.fp8_out ? 1 : 2);
  q.out_b = out.bstride * oesz;
  q.out_g = out.gstride * oesz;
  q.out_p = out.pstride * oesz;
  q.out_P = out.P;
  q.fp32_single = out.fp32_single;
  q.fp8_out = out.fp8_out;
  q.out_scale = L.out_scale;
  q.res = (const char*)out.res;
  const int resz = fp8 ? 1 : 2;
  q.res_b = out.rbstride * resz;
  q.res_g = out.rgstride * resz;
  q.res_p = out.rpstride * resz;
  q.res_P = out.rP ? out.rP : 1;
  q.res_fp8 = fp8 ? 1 : 0;
  q.res_scale = fp8 ? 1.0f / L.out_scale : 1.0f;
  q.err = err;
  const size_t smem = 128 + (size_t)q.a_bytes + (size_t)q.nst * q.sps * q.step_bytes + 8 * (2 + 2 * q.nst) + 8 +
                      8 * (size_t)L.n_steps + 16;
  GW_CHECK_ARG(smem <= 227 * 1024, "shared memory plan too large");
  *smem_out = smem;
  *grid_out = dim3((q.mout0 + 128 * MT - 1) / (128 * MT), B);
}

void launch_conv_tc(const LayerDev& L, const TcIn& in, int lout, const TcOut& out, int B, int* err, cudaStream_t st) {
  TcParams q;
  size_t smem = 0;
  dim3 grid;
  plan_conv_tc(q, L, L.wscale != nullptr, in, lout, out, err, &smem, &grid, B);
  q.wimg = (const char*)L.wq;
  q.table = L.table;
  static bool attr = false;
  if (!attr) {
    GW_CUDA(cudaFuncSetAttribute(conv_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    attr = true;
  }
  conv_tc_kernel<<<grid, kThreads, smem, st>>>(q);
  GW_LAUNCH_CHECK();
}

}  // namespace gw

// Host-only inspection of the lowering and launch plan of one layer (no GPU).
extern "C" int gw_tc_inspect(const int* spec, int precision, const double* wfold, int lin, int in_P, int out_P,
                             void* img_out, size_t img_cap, uint32_t* table_out, int table_cap, int* meta_out) {
  using namespace gw;
  try {
    GW_CHECK_ARG(spec && wfold && img_out && table_out && meta_out, "NULL argument");
    GW_CHECK_ARG(precision == GW_BF16 || precision == GW_FP8, "precision must be BF16 or FP8");
    LayerDev L;
    L.s = LayerSpec{spec[0] != 0, spec[1], spec[2], spec[3], spec[4], spec[5], spec[6], spec[7], true, ACT_NONE};
    const LayerSpec& s = L.s;
    GW_CHECK_ARG(s.cin >= 1 && s.cout >= 1 && s.k >= 1 && s.stride >= 1 && lin >= 1, "bad layer spec");
    std::vector<double> wf(wfold, wfold + (size_t)s.cout * s.cin * s.k);
    std::vector<uint8_t> img;
    std::vector<uint32_t> table;
    std::vector<float> wscale;
    const bool fp8 = precision == GW_FP8;
    lower_layer(L, wf, fp8, img, table, wscale);
    GW_CHECK_ARG(img.size() <= img_cap && (int)table.size() <= table_cap, "output buffers too small");
    memcpy(img_out, img.data(), img.size());
    memcpy(table_out, table.data(), table.size() * 4);
    const int lout = s.lout(lin);
    TcIn in{};
    in.P = in_P;
    in.L = lin;
    TcOut out{};
    out.P = out_P;
    TcParams q;
    size_t smem = 0;
    dim3 grid;
    plan_conv_tc(q, L, fp8, in, lout, out, nullptr, &smem, &grid, 1);
    const int meta[20] = {L.n_steps, L.npad, L.gin, L.pin, L.n_chains, L.dspan, L.dmin, q.MT, q.rows, q.a_bytes,
                          q.sps, q.nst, q.step_bytes, q.ncols, (int)grid.x, q.mout0, q.mout1, (int)q.idesc,
                          (int)smem, lout};
    memcpy(meta_out, meta, sizeof(meta));
    return GW_OK;
  } catch (const gw::Error& e) {
    gw::set_last_error(e.what());
    return e.code;
  }
}

namespace gw {

void launch_to_blocked(const float* x, int64_t xb, int64_t xc, int B, int C, int L, const float* mean,
                       const float* istd, float scale, const TcOut& out, int fp8, cudaStream_t st) {
  const int esz = fp8 ? 1 : 2;
  const int cg = fp8 ? 16 : 8;
  const int64_t total = (int64_t)B * ((C + cg - 1) / cg) * L;
  const int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 32);
  to_blocked_kernel<<<grid, 256, 0, st>>>(x, xb, xc, B, C, L, mean, istd, scale, (char*)out.p, out.bstride * esz,
                                          out.gstride * esz, out.pstride * esz, out.P, fp8);
  GW_LAUNCH_CHECK();
}

void launch_gap_linear_blocked(const TcIn& in, int C, int fp8, float in_scale, const float* w, const float* b,
                               float* out, int B, cudaStream_t st) {
  const int esz = fp8 ? 1 : 2;
  gap_linear_blocked_kernel<<<B, 256, 0, st>>>((const char*)in.p + in.off0 * esz, in.bstride * esz, in.gstride * esz,
                                               in.pstride * esz, in.P, in.L, C, fp8, in_scale, w, b, out);
  GW_LAUNCH_CHECK();
}

}  // namespace gw
