// Per-tile pipeline of the local autoregressive model (device code):
//   gather of the causal context (Eq. 3) -> local network (Section 2.1) ->
//   discretized logistic mixture -> CDF -> 16-bit frequency table.
// Used by the decoder (one wavefront step per tile) and by the encoder (any
// pixels per tile); the arithmetic per pixel is independent of the tile
// position, so both produce identical tables.
#pragma once

#include "nlc_common.cuh"

namespace nlc {

// One pixel slot of a tile.
struct PixSlot {
  int unit;   // unit index, -1 for an empty slot
  int i, j;   // position inside the unit
  int aux;    // decoder: stream index; encoder: pixel index in the batch
};

// ---------------------------------------------------------------------
// Context gather (Eq. 3): taps p enumerate rows dy=-h..-1 with dx=-h..h,
// then dy=0 with dx=-h..-1; feature 3p+c holds channel c.  Outside the
// unit the network input is zero.
// ---------------------------------------------------------------------
__device__ __forceinline__ void tap_offset(int p, int h, int& dy, int& dx) {
  int w = 2 * h + 1;
  dy = p / w - h;
  dx = p % w - h;
}

// FP32 layout: X[f][m] (feature-major), value (2v-255)/255.
template <int MT, bool kCoherent>
__device__ void gather_f32(const Unit* units, const PixSlot* slots, int h, float* X) {
  const int ntap = 2 * h * (h + 1);
  for (int it = threadIdx.x; it < MT * ntap; it += blockDim.x) {
    int m = it % MT, p = it / MT;
    const PixSlot s = slots[m];
    float v0 = 0.f, v1 = 0.f, v2 = 0.f;
    if (s.unit >= 0) {
      const Unit u = units[s.unit];
      int dy, dx;
      tap_offset(p, h, dy, dx);
      int ii = s.i + dy, jj = s.j + dx;
      if (ii >= 0 && ii < u.Hu && jj >= 0 && jj < u.Wu) {
        const uint8_t* px = u.img + ((long long)(u.y0 + ii) * u.img_W + (u.x0 + jj)) * 3;
        int a, b, c;
        if (kCoherent) { a = ld_cg_u8(px); b = ld_cg_u8(px + 1); c = ld_cg_u8(px + 2); }
        else { a = px[0]; b = px[1]; c = px[2]; }
        v0 = __fdiv_rn((float)(2 * a - 255), 255.f);
        v1 = __fdiv_rn((float)(2 * b - 255), 255.f);
        v2 = __fdiv_rn((float)(2 * c - 255), 255.f);
      }
    }
    X[(3 * p + 0) * MT + m] = v0;
    X[(3 * p + 1) * MT + m] = v1;
    X[(3 * p + 2) * MT + m] = v2;
  }
}

__device__ __forceinline__ float elu_f(float x) { return x > 0.f ? x : expm1f(x); }

// ---------------------------------------------------------------------
// FP32 SIMT local network.  Activations are feature-major [n][m]; each
// thread owns 4 pixels x NB outputs (N = 16 NB), accumulating over k in
// ascending order with explicit fma.
// ---------------------------------------------------------------------
enum GemmMode { GM_STORE = 0, GM_ELU = 1, GM_RESID = 2, GM_HEAD = 3 };

template <int MT, int NB, int MODE>
__device__ __noinline__ void gemm_simt(const float* __restrict__ in, int Kd,
                                          const float* __restrict__ WT,
                                          const float* __restrict__ bias, float* __restrict__ out,
                                          int ldp) {
  static_assert(MT == 64, "the SIMT tile is 64 pixels");
  constexpr int N = 16 * NB;
  const int tm = threadIdx.x & 15, tn = threadIdx.x >> 4;
  const int m0 = tm * 4, n0 = tn * NB;
  float acc[4][NB];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < NB; b++) acc[a][b] = 0.f;
  for (int k = 0; k < Kd; k++) {
    const float4 x = *reinterpret_cast<const float4*>(in + k * MT + m0);
    const float* wr = WT + k * N + n0;
    float wv[NB];
#pragma unroll
    for (int b = 0; b < NB; b++) wv[b] = wr[b];
#pragma unroll
    for (int b = 0; b < NB; b++) {
      acc[0][b] = __fmaf_rn(x.x, wv[b], acc[0][b]);
      acc[1][b] = __fmaf_rn(x.y, wv[b], acc[1][b]);
      acc[2][b] = __fmaf_rn(x.z, wv[b], acc[2][b]);
      acc[3][b] = __fmaf_rn(x.w, wv[b], acc[3][b]);
    }
  }
#pragma unroll
  for (int b = 0; b < NB; b++) {
    const float bb = bias[n0 + b];
#pragma unroll
    for (int a = 0; a < 4; a++) {
      float v = __fadd_rn(acc[a][b], bb);
      if (MODE == GM_STORE) out[(n0 + b) * MT + m0 + a] = v;
      if (MODE == GM_ELU) out[(n0 + b) * MT + m0 + a] = elu_f(v);
      if (MODE == GM_RESID) {
        float* o = out + (n0 + b) * MT + m0 + a;
        *o = __fadd_rn(*o, v);
      }
      if (MODE == GM_HEAD) out[(m0 + a) * ldp + n0 + b] = v;
    }
  }
}

template <int MT, int NB>
__device__ __forceinline__ void gemm_layer(int mode, const float* in, int Kd, const float* WT,
                                           const float* bias, float* out, int ldp) {
  switch (mode) {
    case GM_STORE: gemm_simt<MT, NB, GM_STORE>(in, Kd, WT, bias, out, ldp); break;
    case GM_ELU: gemm_simt<MT, NB, GM_ELU>(in, Kd, WT, bias, out, ldp); break;
    case GM_RESID: gemm_simt<MT, NB, GM_RESID>(in, Kd, WT, bias, out, ldp); break;
    default: gemm_simt<MT, NB, GM_HEAD>(in, Kd, WT, bias, out, ldp); break;
  }
}

template <int MT>
__device__ void gemm_dispatch(int mode, const float* in, int Kd, const float* WT, const float* bias,
                              int N, float* out, int ldp) {
  switch (N / 16) {
    case 1: gemm_layer<MT, 1>(mode, in, Kd, WT, bias, out, ldp); break;
    case 2: gemm_layer<MT, 2>(mode, in, Kd, WT, bias, out, ldp); break;
    case 3: gemm_layer<MT, 3>(mode, in, Kd, WT, bias, out, ldp); break;
    case 4: gemm_layer<MT, 4>(mode, in, Kd, WT, bias, out, ldp); break;
    case 5: gemm_layer<MT, 5>(mode, in, Kd, WT, bias, out, ldp); break;
    case 6: gemm_layer<MT, 6>(mode, in, Kd, WT, bias, out, ldp); break;
    case 7: gemm_layer<MT, 7>(mode, in, Kd, WT, bias, out, ldp); break;
    case 8: gemm_layer<MT, 8>(mode, in, Kd, WT, bias, out, ldp); break;
    case 9: gemm_layer<MT, 9>(mode, in, Kd, WT, bias, out, ldp); break;
    default: gemm_layer<MT, 10>(mode, in, Kd, WT, bias, out, ldp); break;
  }
}

// Floats of the packed FP32 weights:
// W0T[F][C] b0[C] {W1T[C][C] b1[C] W2T[C][C] b2[C]} x R WHT[C][NOp] bH[NOp].
__host__ __device__ inline size_t simt_floats(const Dims& d) {
  return (size_t)d.F * d.C + d.C + (size_t)d.R * (2 * d.C * d.C + 2 * d.C) + (size_t)d.C * d.NOp +
         d.NOp;
}

// Shared-memory plan of the FP32 tile pipeline (all offsets in floats).
struct SimtPlan {
  int w_off, a_off, b1_off, u0_off, end;
};

__host__ __device__ inline SimtPlan simt_plan(const Dims& d, int simt_floats, int MT) {
  SimtPlan p;
  int u0 = d.Fp * MT;
  if (d.C * MT > u0) u0 = d.C * MT;
  if (MT * d.ldP > u0) u0 = MT * d.ldP;
  p.w_off = 0;
  p.a_off = (simt_floats + 3) & ~3;
  p.b1_off = p.a_off + d.C * MT;
  p.u0_off = p.b1_off + d.C * MT;
  p.end = p.u0_off + u0;
  return p;
}

// Network of a 64-pixel tile: X (features, in U0) -> P[m][ldP] (in U0).
template <int MT>
__device__ void network_simt_run(const Dims& d, const float* Wt, float* A, float* B1, float* U0) {
  const int C = d.C, F = d.F;
  const float* W0T = Wt;
  const float* b0 = W0T + F * C;
  const float* cur = b0 + C;
  gemm_dispatch<MT>(GM_STORE, U0, F, W0T, b0, C, A, 0);
  __syncthreads();
  for (int r = 0; r < d.R; r++) {
    const float* W1T = cur;
    const float* b1 = W1T + C * C;
    const float* W2T = b1 + C;
    const float* b2 = W2T + C * C;
    cur = b2 + C;
    for (int e = threadIdx.x; e < C * MT; e += blockDim.x) B1[e] = elu_f(A[e]);
    __syncthreads();
    gemm_dispatch<MT>(GM_ELU, B1, C, W1T, b1, C, U0, 0);
    __syncthreads();
    gemm_dispatch<MT>(GM_RESID, U0, C, W2T, b2, C, A, 0);
    __syncthreads();
  }
  for (int e = threadIdx.x; e < C * MT; e += blockDim.x) B1[e] = elu_f(A[e]);
  __syncthreads();
  const float* WHT = cur;
  const float* bH = WHT + C * d.NOp;
  gemm_dispatch<MT>(GM_HEAD, B1, C, WHT, bH, d.NOp, U0, d.ldP);
  __syncthreads();
}

// ---------------------------------------------------------------------
// Discretized logistic mixture and the frequency table of one channel.
// Network outputs of a pixel: [0,K) logits, [K,4K) locations mu_{c,k},
// [4K,7K) log-scales (clamped below at -7), [7K,10K) raw coupling
// coefficients (tanh).  Coupled locations: m_R = mu_R,
// m_G = mu_G + alpha x_R, m_B = mu_B + beta x_R + gamma x_G.
// Boundary b (1..255) sits at e_b = (2b-256)/255; the table is
//   F(b) = sum_k w_k sigmoid((e_b - m_k)/s_k),
//   q_b = clamp(rint(65280 F(b)), 0, 65280), Q_b = max(Q_{b-1}, q_b),
//   cum_b = Q_b + b, cum_256 = 2^16,
// so every frequency is >= 1 and they sum to 2^16.  Component weights:
// R: pi_k; G: prop. to pi_k P_Rk(r); B: prop. to pi_k P_Rk(r) P_Gk(g).
// The device evaluates F so that it is non-decreasing in b (cdf_term
// below); then Q_b = q_b and any cum_b is computed on its own.
// ---------------------------------------------------------------------
constexpr float kInv255 = 1.f / 255.f;
constexpr float kLog2e = 1.4426950408889634f;

// Boundary e_b = (2b - 256)/255 and the scaled value x_v = (2v - 255)/255.
__device__ __forceinline__ float edge_f(int b) { return __fmul_rn((float)(2 * b - 256), kInv255); }
__device__ __forceinline__ float xval_f(int v) { return __fmul_rn((float)(2 * v - 255), kInv255); }

// e^x and log x through the MUFU ex2 / lg2 approximations (deterministic).
__device__ __forceinline__ float exp_f(float x) { return ex2_approx(__fmul_rn(x, kLog2e)); }
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float log_f(float x) { return __fmul_rn(lg2_approx(x), 0.6931471805599453f); }

// softplus(x) = max(x, 0) + log(1 + e^{-|x|})
__device__ __forceinline__ float softplus_f(float x) {
  return __fadd_rn(fmaxf(x, 0.f), log_f(__fadd_rn(1.f, exp_f(-fabsf(x)))));
}
// log(1 - e^{-d}), d > 0.  For d < 1/8 the Taylor series
// 1 - e^{-d} = d (1 - d/2 + d^2/6 - d^3/24 + d^4/120) (relative error below
// 5e-8 there) avoids the cancellation of 1 - e^{-d}.
__device__ __forceinline__ float log1mexp_f(float d) {
  if (d < 0.125f) {
    float p = __fmaf_rn(d, 1.f / 120.f, -1.f / 24.f);
    p = __fmaf_rn(p, d, 1.f / 6.f);
    p = __fmaf_rn(p, d, -0.5f);
    p = __fmaf_rn(p, d, 1.f);
    return log_f(__fmul_rn(d, p));
  }
  return log_f(__fsub_rn(1.f, exp_f(-d)));
}

// log(1 - e^{-d}) of a component with log-scale ls and inv = e^{-ls}, where
// d = (2/255) inv is the bin width over the scale; for d < e^-14 it is taken
// as log d = log(2/255) - ls (error O(d)), which stays finite when inv
// underflows.
__device__ __forceinline__ float bin_log_width(float ls, float inv) {
  const float logd = __fsub_rn(-4.848116f, ls);
  return logd < -14.f ? logd : log1mexp_f(__fmul_rn(2.f * kInv255, inv));
}

// tanh x = sign(x) (1 - 2/(1 + e^{2|x|})), |x| capped at 20 (tanh = 1 in FP32).
__device__ __forceinline__ float tanh_f(float x) {
  const float ax = fminf(fabsf(x), 20.f);
  const float r = rcp_approx(__fadd_rn(1.f, exp_f(__fmul_rn(2.f, ax))));
  return copysignf(__fsub_rn(1.f, __fmul_rn(2.f, r)), x);
}

// log P(v) of one logistic component with location m, inv = e^{-ls} and
// lme = bin_log_width(ls, inv), stable in both tails:
// log P = -softplus(-a) - softplus(b) + log(1 - e^{-(a-b)}), a - b = (2/255)/s.
__device__ __forceinline__ float log_bin_mass_f(float m, float inv, float lme, int v) {
  if (v <= 0) return -softplus_f(-__fmul_rn(__fsub_rn(edge_f(1), m), inv));
  if (v >= 255) return -softplus_f(__fmul_rn(__fsub_rn(edge_f(255), m), inv));
  const float a = __fmul_rn(__fsub_rn(edge_f(v + 1), m), inv);
  const float b = __fmul_rn(__fsub_rn(edge_f(v), m), inv);
  return __fadd_rn(__fsub_rn(-softplus_f(-a), softplus_f(b)), lme);
}

// Scratch of one coding group (a warp, or half a warp) in the CDF stage:
// the channel's active components (weight >= kWmin), compacted in
// increasing component order, as (m_k, c_k = log2(e)/s_k, w_k 2^23, 0),
// then zero entries (weight 0, term 0) up to 2 kMaxK, so that unrolled
// loops may read past the last active component.
struct alignas(16) WarpScratch {
  float4 cp[2 * kMaxK];
  float4 pad;  // 528-byte stride: the two groups of a warp read different banks
};

// Table of one coding warp for decoding with an explicit cum[0..255]
// (lane-interleaved, see cum_pos); cum_256 = 2^16.
struct TableScratch {
  uint32_t cum[256];
};

// Components whose weight is below 2^-17 are left out of the CDF: together
// they move 65280 F(b) by at most half a count per component.
constexpr float kWmin = 7.62939453125e-06f;

// Bound of a component's location in the CDF (2^100; |m - e| c stays finite).
constexpr float kMMax = 1.2676506002282294e30f;

// Fixed point with 23 fraction bits: x in [0, 2^23] plus 2^23, rounded to
// nearest, is 2^23 + rint(x) (the spacing of floats in [2^23, 2^24] is 1);
// its bit pattern minus that of 2^23 is rint(x).
constexpr float kFixOne = 8388608.f;           // 2^23
constexpr uint32_t kFixOneBits = 0x4B000000u;  // bit pattern of 2^23
constexpr float kLn2x23 = 15.942385152878742f;  // 23 ln 2

// rint(e 2^23) for e in [0, 1].
__device__ __forceinline__ uint32_t fix23(float e) {
  return (uint32_t)__float_as_int(__fadd_rn(__fmul_rn(e, kFixOne), kFixOne)) - kFixOneBits;
}

// ---------------------------------------------------------------------
// Coding groups.  One pixel's channels are coded by a group of GW lanes
// (GW = 32: a whole warp; GW = 16: half a warp, so that a warp codes two
// pixels at once); lanes gl < K of a group hold component gl.  Group
// reductions over floats are xor butterflies, which give the same value in
// every lane of the group and, for K <= 16, the same value for GW = 16 and
// GW = 32 (the upper half adds exact zeros first).
// ---------------------------------------------------------------------
template <int GW>
__device__ __forceinline__ float grp_max(float v) {
#pragma unroll
  for (int o = GW / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o, GW));
  return v;
}
template <int GW>
__device__ __forceinline__ float grp_sum(float v) {
#pragma unroll
  for (int o = GW / 2; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o, GW));
  return v;
}
template <int GW>
__device__ __forceinline__ unsigned grp_mask(int lane) {
  return GW == 32 ? 0xffffffffu : (0xFFFFu << (lane & 16));
}
// Exact group maximum of floats and exact group sum of integers.  A whole
// warp uses redux.sync (the maximum on order-preserving integer keys:
// negative floats get their magnitude bits flipped); a 16-lane group uses
// xor butterflies, because redux.sync with a mask per half warp is slower
// than the butterfly.  Both forms give the same value for inputs that are
// not NaN (the integer keys would rank a NaN above +inf, fmaxf drops it), so
// the callers map NaN to -inf first (no_nan).
template <int GW>
__device__ __forceinline__ float grp_max_r(float v) {
  if constexpr (GW == 32) {
    int k = __float_as_int(v);
    k = k >= 0 ? k : k ^ 0x7FFFFFFF;
    k = __reduce_max_sync(0xffffffffu, k);
    return __int_as_float(k >= 0 ? k : k ^ 0x7FFFFFFF);
  } else {
    return grp_max<GW>(v);
  }
}
__device__ __forceinline__ float no_nan(float v) { return v == v ? v : -INFINITY; }
template <int GW>
__device__ __forceinline__ uint32_t grp_isum(uint32_t v) {
  if constexpr (GW == 32) {
    return __reduce_add_sync(0xffffffffu, v);
  } else {
#pragma unroll
    for (int o = GW / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, GW);
    return v;
  }
}
// The group's bits of a warp ballot, group lane 0 in bit 0.
template <int GW>
__device__ __forceinline__ unsigned grp_ballot(bool p) {
  const unsigned b = __ballot_sync(0xffffffffu, p);
  return GW == 32 ? b : ((b >> (threadIdx.x & 16)) & 0xFFFFu);
}

// Position of cum_b (b < 256) in TableScratch::cum for groups of GW lanes:
// lane gl's boundaries b = BPL gl + q sit at q GW + gl, so the group's
// stores and loads of one q hit consecutive banks.
template <int GW>
__device__ __forceinline__ int cum_pos(int b) {
  constexpr int BPL = 256 / GW;
  return (b % BPL) * GW + b / BPL;
}
template <int GW>
__device__ __forceinline__ uint32_t cum_at(const TableScratch& ws, int b) {
  return b >= 256 ? 65536u : ws.cum[cum_pos<GW>(b)];
}

// Per-pixel mixture state held by lane k (< K) for component k.
struct CompState {
  float logpi, lw;      // log pi_k, running log weight
  float mu[3], co[3];   // locations, coupling coefficients (tanh)
  float inv[3];         // 1/s = e^{-ls} (log-scale ls clamped at -7)
  float c[3];           // log2(e) / s
  float lme[3];         // bin_log_width(ls, 1/s)
};

template <int GW = 32>
__device__ __forceinline__ void comp_init(const float* P, int K, int gl, CompState& cs) {
  // log-sum-exp of the logits: exact max, then the sum of e^{logit - max}
  // in fixed point (an exact integer sum, S >= 2^23 from the max itself)
  const float logit = gl < K ? no_nan(P[gl]) : -INFINITY;  // a NaN logit: weight 0
  const float mx = grp_max_r<GW>(logit);
  const uint32_t E = fix23(gl < K ? exp_f(__fsub_rn(logit, mx)) : 0.f);
  const uint32_t S = grp_isum<GW>(E);
  const float lse = __fadd_rn(mx, __fsub_rn(log_f((float)S), kLn2x23));
  cs.logpi = __fsub_rn(logit, lse);
  cs.lw = cs.logpi;
  if (gl < K) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
      cs.mu[c] = P[K + c * K + gl];
      const float ls = fmaxf(P[4 * K + c * K + gl], -7.f);
      cs.co[c] = tanh_f(P[7 * K + c * K + gl]);
      cs.inv[c] = exp_f(-ls);
      cs.c[c] = __fmul_rn(cs.inv[c], kLog2e);
      cs.lme[c] = bin_log_width(ls, cs.inv[c]);
    }
  }
}

// a[ch] by selects (ch need not be a compile-time constant, so the arrays
// stay in registers when the channel loop is not unrolled).
template <class T>
__device__ __forceinline__ T pick3(const T (&a)[3], int ch) {
  return ch == 0 ? a[0] : (ch == 1 ? a[1] : a[2]);
}

// Location of channel ch of component (lane) given decoded r, g.
__device__ __forceinline__ float comp_mean(const CompState& cs, int ch, int r, int g) {
  const float xr = xval_f(r), xg = xval_f(g);
  if (ch == 0) return cs.mu[0];
  if (ch == 1) return __fadd_rn(cs.mu[1], __fmul_rn(cs.co[0], xr));
  return __fadd_rn(__fadd_rn(cs.mu[2], __fmul_rn(cs.co[1], xr)), __fmul_rn(cs.co[2], xg));
}

// ---------------------------------------------------------------------
// Pointwise quantised CDF.  F(b) is a fixed-point number in units of 2^-23:
// the sum over the active components of rint(w_k 2^23 sigmoid((e_b-m_k)/s_k)).
// Every operation from b to a term is non-decreasing in b: correctly
// rounded arithmetic with fixed operands, rint, and the MUFU approximations
// ex2.approx (over all floats, saturating to +0 and +inf) and rcp.approx (on
// [1, +inf]), which are monotone on sm_103 (checked exhaustively over those
// ranges by the library before a context is created, see
// mono_check_kernel).  So F is non-decreasing in b as computed, the running
// max of the quantiser leaves q unchanged, and each cum_b follows from b
// alone.  Integer sums do not depend on the order of their terms: every
// split of the components over lanes, in the encoder, the decoder or the
// table entry point, gives the same cum_b.
// ---------------------------------------------------------------------

// One component's term of F at boundary value e: the logistic is
// 1/(1 + 2^z) with z = (m - e) log2(e)/s (a z beyond the float range of 2^z
// gives 2^z = +inf or +0, hence the term's limits 0 and w), and the fused
// w sigmoid + 2^23, rounded once to nearest, is 2^23 + rint(w 2^23 sigmoid)
// (w 2^23 sigmoid lies in [0, 2^23], float spacing 1 in [2^23, 2^24]), read
// back from its bits.  kClamp clamps z to [-126, 126] first, which changes no
// term: past 126 the term is 0 and below -126 it is rint(w) either way
// (1 + 2^z rounds to 1).  The whole-warp search, one pixel per warp and bound
// by latency, measured faster with the clamp; the 16-lane search, bound by
// throughput, without it.
template <bool kClamp = false>
__device__ __forceinline__ uint32_t cdf_term(float e, const float4& p) {
  float z = __fmul_rn(__fsub_rn(p.x, e), p.y);
  if (kClamp) z = fminf(fmaxf(z, -126.f), 126.f);
  const float y = __fmaf_rn(p.z, rcp_approx(__fadd_rn(1.f, ex2_approx(z))), kFixOne);
  return (uint32_t)__float_as_int(y) - kFixOneBits;
}

// Partial fixed-point F at boundary value e over components i0, i0 + di, ...
// (di <= 4), five independent terms at a time (the K = 10 mixture in two
// rounds); entries past the active ones are zero, so the reads stay below
// nact - 1 + 4 di + 1 <= 32 entries.  (Handling the remainder exactly
// instead of padding it measured slower: the larger code costs more than
// the skipped terms.)
template <bool kClamp = false>
__device__ __forceinline__ uint32_t cdf_fix(const WarpScratch& ws, int nact, float e, int i0,
                                            int di) {
  uint32_t F = 0;
  for (int i = i0; i < nact; i += 5 * di) {
    const uint32_t t0 = cdf_term<kClamp>(e, ws.cp[i]);
    const uint32_t t1 = cdf_term<kClamp>(e, ws.cp[i + di]);
    const uint32_t t2 = cdf_term<kClamp>(e, ws.cp[i + 2 * di]);
    const uint32_t t3 = cdf_term<kClamp>(e, ws.cp[i + 3 * di]);
    const uint32_t t4 = cdf_term<kClamp>(e, ws.cp[i + 4 * di]);
    F += ((t0 + t1) + (t2 + t3)) + t4;
  }
  return F;
}

// cum_b = q_b + b with q_b = clamp(rint(65280 F), 0, 65280), F = Fi 2^-23
// (ties to even); cum_0 = 0 and cum_256 = 2^16.
__device__ __forceinline__ uint32_t cum_fix(uint32_t Fi, int b) {
  if (b <= 0) return 0u;
  if (b >= 256) return 65536u;
  const unsigned long long P = (unsigned long long)Fi * (unsigned long long)kMq;
  uint32_t q = (uint32_t)(P >> 23);
  const uint32_t r = (uint32_t)(P & 0x7FFFFFull);
  q += (r > 0x400000u || (r == 0x400000u && (q & 1u))) ? 1u : 0u;
  return (q < (uint32_t)kMq ? q : (uint32_t)kMq) + (uint32_t)b;
}

// Channel ch of the pixel: component weights (softmax of the running log
// weights) and locations, compacted into ws.cp.  Returns the location of the
// lane's component (for the posterior update); nact = active components.
template <int GW>
__device__ __forceinline__ float channel_setup(const CompState& cs, int K, int ch, int r, int g,
                                               int gl, WarpScratch& ws, int& nact) {
  // w_k 2^23: for R the mixture weights pi_k = e^{log pi_k} (normalised by
  // comp_init); for G and B the posterior e^{lw_k - max} / sum, the sum taken
  // exactly in fixed point
  float wS = 0.f;
  if (ch == 0) {
    if (gl < K) wS = __fmul_rn(fminf(exp_f(cs.logpi), 1.f), kFixOne);
  } else {
    const float lw = gl < K ? no_nan(cs.lw) : -INFINITY;
    const float mx = grp_max_r<GW>(lw);
    const uint32_t E = fix23(gl < K ? exp_f(__fsub_rn(lw, mx)) : 0.f);
    const uint32_t S = grp_isum<GW>(E);
    wS = fminf(__fmul_rn((float)E, __fmul_rn(kFixOne, rcp_approx((float)S))), kFixOne);
  }
  // the location within +-2^100 (a NaN network output becomes -2^100), so
  // that every term is a number: past |m| = 2^100 the CDF is a step either way
  const float m = gl < K ? fminf(fmaxf(comp_mean(cs, ch, r, g), -kMMax), kMMax) : 0.f;
  // the weights sum to one, so at least one component is active
  const bool on = gl < K && wS >= kWmin * kFixOne;
  const unsigned bits = grp_ballot<GW>(on);
  nact = __popc(bits);
  for (int p = gl; p < 2 * kMaxK; p += GW)
    if (p >= nact) ws.cp[p] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (on) ws.cp[__popc(bits & ((1u << gl) - 1u))] = make_float4(m, pick3(cs.c, ch), wS, 0.f);
  __syncwarp();
  return m;
}

// Decoder's symbol search for slot in [0, 2^16): s with cum_s <= slot <
// cum_{s+1}, and those two values.  Round 1: lane gl evaluates cum at
// b = B (gl + 1) (B = 256/GW; the last lane holds cum_256); the count c of
// those <= slot locates s in [B c, B c + B).  Round 2: the B - 1 boundaries
// inside, with the components split over the GW/B lanes that share one.
template <int GW>
__device__ __forceinline__ int cdf_search(const WarpScratch& ws, int nact, uint32_t slot, int gl,
                                          uint32_t& c0, uint32_t& c1) {
  constexpr int B = 256 / GW;
  constexpr int P = GW / B;
  const unsigned full = 0xffffffffu;
  uint32_t u1 = 65536u;
  if (gl < GW - 1) {
    const int b = B * (gl + 1);
    u1 = cum_fix(cdf_fix<GW == 32>(ws, nact, edge_f(b), 0, 1), b);
  }
  const int c = __popc(grp_ballot<GW>(u1 <= slot));
  const int j = gl % B, part = gl / B;
  const int b2 = B * c + j + 1;
  uint32_t F2 = 0;
  if (j < B - 1) F2 = cdf_fix<GW == 32>(ws, nact, edge_f(b2), part, P);
#pragma unroll
  for (int o = B; o < GW; o <<= 1) F2 += __shfl_xor_sync(full, F2, o, GW);
  const uint32_t top = __shfl_sync(full, u1, c, GW);  // cum_{B (c+1)}
  const uint32_t u2 = j < B - 1 ? cum_fix(F2, b2) : top;
  const int c2 = __popc(grp_ballot<GW>(part == 0 && u2 <= slot));
  c1 = __shfl_sync(full, u2, c2, GW);
  const uint32_t lo2 = __shfl_sync(full, u2, c2 > 0 ? c2 - 1 : 0, GW);
  const uint32_t lo1 = __shfl_sync(full, u1, c > 0 ? c - 1 : 0, GW);
  c0 = c2 > 0 ? lo2 : (c > 0 ? lo1 : 0u);
  return B * c + c2;
}

// Encoder's pair cum_v, cum_{v+1}: lanes of even / odd gl evaluate b = v /
// v + 1 over components gl/2 and gl/2 + GW/2 (K <= 16: every component once).
template <int GW>
__device__ __forceinline__ void cdf_pair(const WarpScratch& ws, int v, int gl, uint32_t& c0,
                                         uint32_t& c1) {
  const unsigned full = 0xffffffffu;
  const int b = v + (gl & 1);
  const float e = edge_f(b);
  uint32_t F = cdf_term(e, ws.cp[gl >> 1]) + cdf_term(e, ws.cp[(gl >> 1) + GW / 2]);
#pragma unroll
  for (int o = 2; o < GW; o <<= 1) F += __shfl_xor_sync(full, F, o, GW);
  const uint32_t u = cum_fix(F, b);
  c0 = __shfl_sync(full, u, 0, GW);
  c1 = __shfl_sync(full, u, 1, GW);
}

// Symbol s with cum_s <= slot < cum_{s+1} in an explicit table.
template <int GW>
__device__ __forceinline__ int table_search(const TableScratch& ws, uint32_t slot, int lane) {
  constexpr int BPL = 256 / GW;
  const int gl = lane & (GW - 1);
  int cnt = 0;
#pragma unroll
  for (int q = 0; q < BPL; q++) {
    const int b = gl * BPL + q;
    cnt += (b >= 1 && ws.cum[q * GW + gl] <= slot) ? 1 : 0;
  }
  return __reduce_add_sync(grp_mask<GW>(lane), cnt);
}

// Posterior update after channel ch took value v (lanes < K).
__device__ __forceinline__ void comp_observe(CompState& cs, int K, int ch, float m, int v, int gl) {
  if (gl < K) cs.lw = __fadd_rn(cs.lw, log_bin_mass_f(m, pick3(cs.inv, ch), pick3(cs.lme, ch), v));
}

}  // namespace nlc
