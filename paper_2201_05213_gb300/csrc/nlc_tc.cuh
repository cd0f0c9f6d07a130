// BF16 local network on the 5th-generation tensor cores (tcgen05 + TMEM).
//
// A tile is M = 128 pixels.  Each layer is one chain of
// tcgen05.mma.cta_group::1.kind::f16 instructions (K = 16 per instruction,
// FP32 accumulation in TMEM) issued by one thread; the accumulator is read
// back with tcgen05.ld by all 8 warps (warp w reads TMEM lanes 32(w%4)..+31
// and half w/4 of the columns), bias/ELU/residual are applied in registers
// and the next layer's A operand is written to shared memory as BF16 in the
// canonical no-swizzle K-major layout:
//   element (r, k) of an R x Kd matrix at
//   ((r/8) * (Kd/8) + k/8) * 64 + (r%8) * 8 + (k%8)   (BF16 elements)
// i.e. 8x8 core matrices of 128 contiguous bytes; the leading-dimension byte
// offset (next core matrix along K) is 128 and the stride-dimension byte
// offset (next 8-row group) is Kd/8 * 128.
//
// Network input: the integer 2v-255 (exact in BF16); the 1/255 of the scaled
// pixel value (2v-255)/255 is folded into the first-layer weights.  The
// residual stream stays in FP32 registers; only layer inputs are BF16.
#pragma once

#include <cuda_bf16.h>

#include "nlc_common.cuh"
#include "nlc_model.cuh"

namespace nlc {

constexpr int kTcM = 128;
constexpr int kTileMax = 128;
constexpr int kTmemCols = 128;
constexpr unsigned kMbarSpin = 1u << 22;

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

struct TcPlan {
  int w0, w1[kMaxR], w2[kMaxR], wh, bias, hbuf, p, mbar, tslot, end;
};

__host__ __device__ inline TcPlan tc_plan(const Dims& d) {
  TcPlan p;
  int o = 0;
  p.w0 = o;
  o += d.C * d.Fp * 2;
  for (int r = 0; r < kMaxR; r++) {
    p.w1[r] = o;
    if (r < d.R) o += d.C * d.C * 2;
    p.w2[r] = o;
    if (r < d.R) o += d.C * d.C * 2;
  }
  p.wh = o;
  o += d.NOp * d.C * 2;
  p.bias = o;
  o += (d.C + 2 * d.R * d.C + d.NOp) * 4;
  o = align_up(o, 128);
  p.hbuf = o;
  o += kTcM * d.C * 2;
  o = align_up(o, 128);
  p.p = o;  // P[m][ldP] FP32, aliased with the BF16 context tile X
  int pbytes = kTcM * d.ldP * 4, xbytes = kTcM * d.Fp * 2;
  o += pbytes > xbytes ? pbytes : xbytes;
  o = align_up(o, 16);
  p.mbar = o;
  o += 8;
  p.tslot = o;
  o += 8;
  p.end = align_up(o, 128);
  return p;
}

__host__ __device__ inline size_t tc_smem_bytes(const Dims& d) { return (size_t)tc_plan(d).end; }
__host__ __device__ inline size_t umma_halves(const Dims& d) {
  return (size_t)d.C * d.Fp + 2 * (size_t)d.R * d.C * d.C + (size_t)d.NOp * d.C;
}
__host__ __device__ inline size_t bias_floats(const Dims& d) { return (size_t)d.C + 2 * (size_t)d.R * d.C + d.NOp; }

struct TcSmem {
  unsigned char* base;
  uint16_t* X;
  uint16_t* H;
  float* P;
  float* bias;
  uint64_t* mbar;
  uint32_t* tslot;
  uint32_t tmem;
  uint32_t phase;
  int ok;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__host__ __device__ __forceinline__ int umma_off(int r, int k, int Kd) {
  return ((r >> 3) * (Kd >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ TcSmem tc_carve(const Dims& d, unsigned char* smem) {
  TcPlan p = tc_plan(d);
  TcSmem t;
  t.base = smem;
  t.X = reinterpret_cast<uint16_t*>(smem + p.p);
  t.H = reinterpret_cast<uint16_t*>(smem + p.hbuf);
  t.P = reinterpret_cast<float*>(smem + p.p);
  t.bias = reinterpret_cast<float*>(smem + p.bias);
  t.mbar = reinterpret_cast<uint64_t*>(smem + p.mbar);
  t.tslot = reinterpret_cast<uint32_t*>(smem + p.tslot);
  t.tmem = 0;
  t.phase = 0;
  t.ok = 1;
  return t;
}

// --- PTX wrappers --------------------------------------------------------
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;                // base offset 0, relative LBO, no swizzle
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtm),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(mbar))
      : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t phase) {
  for (unsigned it = 0; it < kMbarSpin; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 8 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
      : "r"(taddr)
      : "memory");
  v[0] = __uint_as_float(r0);
  v[1] = __uint_as_float(r1);
  v[2] = __uint_as_float(r2);
  v[3] = __uint_as_float(r3);
  v[4] = __uint_as_float(r4);
  v[5] = __uint_as_float(r5);
  v[6] = __uint_as_float(r6);
  v[7] = __uint_as_float(r7);
}

// 32 consecutive FP32 columns of this thread's TMEM lane (one load, one wait).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

// The columns c0 .. c0 + ch - 1 (ch = 8, 16, 24 or 32) of this thread's lane.
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, int ch, float (&v)[32]) {
  if (ch == 32) {
    tmem_ld32(taddr, v);
  } else {
#pragma unroll
    for (int g = 0; g < 4; g++) {
      if (g < ch / 8) {
        float u[8];
        tmem_ld8(taddr + (uint32_t)(8 * g), u);
#pragma unroll
        for (int e = 0; e < 8; e++) v[8 * g + e] = u[e];
      }
    }
  }
}

// --- setup / teardown -------------------------------------------------------
__device__ __forceinline__ void tc_setup(TcSmem& t) {
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(t.mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(t.tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  t.tmem = *t.tslot;
  t.phase = 0;
  t.ok = 1;
}

__device__ __forceinline__ void tc_teardown(TcSmem& t) {
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(t.tmem),
                 "r"(kTmemCols)
                 : "memory");
}

__device__ __forceinline__ void tc_load_weights(const Dims& d, const WeightView& w, TcSmem& t) {
  const int nh = w.umma_halves;  // multiple of 64 (core matrices)
  const uint4* src = reinterpret_cast<const uint4*>(w.umma);
  uint4* dst = reinterpret_cast<uint4*>(t.base);
  for (int i = threadIdx.x; i < nh / 8; i += blockDim.x) dst[i] = src[i];
  const int nb = (int)bias_floats(d);
  for (int i = threadIdx.x; i < nb; i += blockDim.x) t.bias[i] = w.bias[i];
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat16 x = __float2bfloat16_rn(a), y = __float2bfloat16_rn(b);
  return (uint32_t)__bfloat16_as_ushort(x) | ((uint32_t)__bfloat16_as_ushort(y) << 16);
}

// --- gather ------------------------------------------------------------------
// X(m, k) = 2v - 255 for feature k = 3p + c of tap p, 0 outside the unit,
// for k >= F and for empty slots.  Each thread writes 16-byte chunks.
template <bool kCoherent>
__device__ __noinline__ void tc_gather(const Unit* units, const PixSlot* slots, const Dims& d,
                                       TcSmem& t, int n_valid) {
  // (pixel, tap) pairs of the valid rows; each thread issues all its context
  // loads before any shared-memory store.  Rows >= n_valid are left as they
  // are: tensor-core rows are independent and their outputs are not read.
  constexpr int kMaxPairs = (kTcM * 2 * kMaxH * (kMaxH + 1) + kThreads - 1) / kThreads;
  const int Fp = d.Fp, F = d.F, h = d.h, w2 = 2 * h + 1, ntap = 2 * h * (h + 1);
  const int npairs = n_valid * ntap;
  uint32_t val[kMaxPairs];
#pragma unroll
  for (int r = 0; r < kMaxPairs; r++) {
    const int it = threadIdx.x + r * kThreads;
    uint32_t v = 0;
    if (it < npairs) {
      const int m = it / ntap, p = it - m * ntap;
      const PixSlot s = slots[m];
      const Unit u = units[s.unit];
      const int ii = s.i + p / w2 - h, jj = s.j + p % w2 - h;
      if (ii >= 0 && ii < u.Hu && jj >= 0 && jj < u.Wu) {
        const uint8_t* px = u.img + ((long long)(u.y0 + ii) * u.img_W + (u.x0 + jj)) * 3;
        const uint32_t b0 = kCoherent ? ld_cg_u8(px) : px[0];
        const uint32_t b1 = kCoherent ? ld_cg_u8(px + 1) : px[1];
        const uint32_t b2 = kCoherent ? ld_cg_u8(px + 2) : px[2];
        v = b0 | (b1 << 8) | (b2 << 16) | (1u << 24);
      }
    }
    val[r] = v;
  }
#pragma unroll
  for (int r = 0; r < kMaxPairs; r++) {
    const int it = threadIdx.x + r * kThreads;
    if (it < npairs) {
      const int m = it / ntap, p = it - m * ntap;
      const uint32_t v = val[r];
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const float x = (v >> 24) ? (float)(2 * (int)((v >> (8 * c)) & 0xFFu) - 255) : 0.f;
        t.X[umma_off(m, 3 * p + c, Fp)] = __bfloat16_as_ushort(__float2bfloat16_rn(x));
      }
    }
  }
  const int npad = Fp - F;
  for (int it = threadIdx.x; it < n_valid * npad; it += kThreads) {
    const int m = it / npad, k = F + it % npad;
    t.X[umma_off(m, k, Fp)] = 0;
  }
}

// --- network -----------------------------------------------------------------
__device__ __forceinline__ void tc_issue(const TcSmem& t, uint32_t a_off, uint32_t b_off, int Kd,
                                         int N) {
  if (threadIdx.x == 0) {
    fence_after_sync();
    const uint32_t a0 = smem_u32(t.base + a_off), b0 = smem_u32(t.base + b_off);
    const uint32_t sbo = (uint32_t)(Kd / 8) * 128u;
    const uint32_t idesc = idesc_bf16(kTcM, N);
    for (int s = 0; s < Kd / 16; s++) {
      mma_bf16(t.tmem, umma_desc(a0 + 256u * s, 128u, sbo), umma_desc(b0 + 256u * s, 128u, sbo),
               idesc, s > 0 ? 1u : 0u);
    }
    mma_commit(t.mbar);
  }
}

__device__ __forceinline__ bool tc_wait(TcSmem& t) {
  bool ok = mbar_wait(t.mbar, t.phase);
  t.phase ^= 1u;
  fence_after_sync();
  return ok;
}

__device__ __forceinline__ float elu_tc(float x) {
  return x > 0.f ? x : __fsub_rn(ex2_approx(__fmul_rn(x, 1.4426950408889634f)), 1.f);
}

// Writes 8 values (columns k0..k0+7) of row r into the BF16 H tile.
__device__ __forceinline__ void store_h8(uint16_t* H, int r, int k0, int C, const float (&v)[8]) {
  uint4 q;
  q.x = pack_bf16(v[0], v[1]);
  q.y = pack_bf16(v[2], v[3]);
  q.z = pack_bf16(v[4], v[5]);
  q.w = pack_bf16(v[6], v[7]);
  *reinterpret_cast<uint4*>(H + umma_off(r, k0, C)) = q;
}

// Runs the whole network on the tile in X; P[m][ldP] = head outputs.
static __device__ __noinline__ bool tc_network(const Dims& d, TcSmem& t, int n_valid) {
  const TcPlan pl = tc_plan(d);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = 32 * (warp & 3) + lane;
  // a warp whose 32 TMEM lanes hold no valid pixel skips its epilogue
  const bool live = 32 * (warp & 3) < n_valid;
  const int half = warp >> 2;
  const uint32_t tl = t.tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  const int C = d.C, ch = C / 2, c0 = half * ch;
  const float* b0 = t.bias;
  float a[kMaxC / 2];
  bool ok = true;

  // layer 0: a = X W0^T + b0, H = ELU(a)
  fence_async_smem();
  __syncthreads();
  tc_issue(t, (uint32_t)pl.p, (uint32_t)pl.w0, d.Fp, C);
  ok &= tc_wait(t);
  if (live) {
    float v[32];
    tmem_ld_cols(tl + (uint32_t)c0, ch, v);
#pragma unroll
    for (int g = 0; g < kMaxC / 16; g++) {
      if (g < ch / 8) {
        float u[8];
#pragma unroll
        for (int e = 0; e < 8; e++) {
          a[8 * g + e] = __fadd_rn(v[8 * g + e], b0[c0 + 8 * g + e]);
          u[e] = elu_tc(a[8 * g + e]);
        }
        store_h8(t.H, row, c0 + 8 * g, C, u);
      }
    }
  }
  fence_before_sync();
  fence_async_smem();
  __syncthreads();

  for (int r = 0; r < d.R; r++) {
    const float* b1 = t.bias + C + 2 * r * C;
    const float* b2 = b1 + C;
    // hidden = ELU(H W1^T + b1)
    tc_issue(t, (uint32_t)pl.hbuf, (uint32_t)pl.w1[r], C, C);
    ok &= tc_wait(t);
    if (live) {
      float v[32];
      tmem_ld_cols(tl + (uint32_t)c0, ch, v);
#pragma unroll
      for (int g = 0; g < kMaxC / 16; g++) {
        if (g < ch / 8) {
          float u[8];
#pragma unroll
          for (int e = 0; e < 8; e++) u[e] = elu_tc(__fadd_rn(v[8 * g + e], b1[c0 + 8 * g + e]));
          store_h8(t.H, row, c0 + 8 * g, C, u);
        }
      }
    }
    fence_before_sync();
    fence_async_smem();
    __syncthreads();
    // a += H W2^T + b2, H = ELU(a)
    tc_issue(t, (uint32_t)pl.hbuf, (uint32_t)pl.w2[r], C, C);
    ok &= tc_wait(t);
    if (live) {
      float v[32];
      tmem_ld_cols(tl + (uint32_t)c0, ch, v);
#pragma unroll
      for (int g = 0; g < kMaxC / 16; g++) {
        if (g < ch / 8) {
          float u[8];
#pragma unroll
          for (int e = 0; e < 8; e++) {
            a[8 * g + e] = __fadd_rn(a[8 * g + e], __fadd_rn(v[8 * g + e], b2[c0 + 8 * g + e]));
            u[e] = elu_tc(a[8 * g + e]);
          }
          store_h8(t.H, row, c0 + 8 * g, C, u);
        }
      }
    }
    fence_before_sync();
    fence_async_smem();
    __syncthreads();
  }

  // head: P = H WH^T + bH
  const float* bh = t.bias + C + 2 * d.R * C;
  tc_issue(t, (uint32_t)pl.hbuf, (uint32_t)pl.wh, C, d.NOp);
  ok &= tc_wait(t);
  const int nh = d.NOp / 2, n0 = half * nh;
  if (live) {
    // columns n0 .. n0 + nh - 1 in loads of up to 32 columns
    for (int c = 0; c < nh; c += 32) {
      const int cw = nh - c < 32 ? nh - c : 32;
      float v[32];
      if (cw == 32) {
        tmem_ld32(tl + (uint32_t)(n0 + c), v);
      } else {
        tmem_ld_cols(tl + (uint32_t)(n0 + c), cw & ~7, v);
      }
      float* o = t.P + (size_t)row * d.ldP + n0 + c;
#pragma unroll
      for (int e = 0; e < 32; e++)
        if (e < (cw & ~7)) o[e] = __fadd_rn(v[e], bh[n0 + c + e]);
    }
  }
  fence_before_sync();
  __syncthreads();
  return __syncthreads_and(ok ? 1 : 0) != 0;
}

cudaError_t launch_repack_umma(const Dims& d, const float* w, uint16_t* umma, float* bias,
                               cudaStream_t s);

}  // namespace nlc
