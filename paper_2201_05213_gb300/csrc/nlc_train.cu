// Maximum-likelihood training of the local model (Eq. 2): one fused kernel
// runs, per 64-pixel tile, the forward pass, the mixture NLL with its
// analytic gradient, and the adjoint of the 1x1 residual blocks and of the
// masked first layer; weight gradients accumulate in a per-CTA slot that a
// second kernel reduces in a fixed order (deterministic).
#include <cuda_runtime.h>
#include <stdint.h>

#include "nlc_common.cuh"
#include "nlc_model.cuh"
#include "nlc_train.cuh"

namespace nlc {

constexpr int kTM = 64;

struct TrainPlan {
  int X, A, Hp, P, DP, T1, T2, XP, zeros, red, ldx, end;  // float offsets
};

__host__ __device__ inline TrainPlan train_plan(const Dims& d) {
  TrainPlan p;
  int o = 0;
  p.ldx = (d.Fp > d.C ? d.Fp : d.C) + 4;
  p.X = o; o += d.Fp * kTM;
  p.A = o; o += (d.R + 1) * d.C * kTM;
  p.Hp = o; o += d.R * d.C * kTM;
  p.P = o; o += kTM * d.ldP;
  p.DP = o; o += d.NOp * kTM;
  p.T1 = o; o += d.C * kTM;
  p.T2 = o; o += d.C * kTM;
  p.XP = o; o += kTM * p.ldx;
  p.zeros = o; o += (d.NOp > d.C ? d.NOp : d.C);
  p.red = o; o += 32;
  p.end = o;
  return p;
}

__host__ __device__ inline size_t train_smem_bytes(const Dims& d) {
  return (size_t)train_plan(d).end * 4 + sizeof(PixSlot) * kTM;
}

__device__ __forceinline__ float elu_d(float x) { return x > 0.f ? 1.f : expf(x); }

// x(m, k) pixel-major copy of a feature-major [rows][64] tile.
__device__ __forceinline__ void to_pixel_major(const float* src, int rows, float* dst, int ldx) {
  for (int e = threadIdx.x; e < rows * kTM; e += blockDim.x) {
    const int r = e / kTM, m = e % kTM;
    dst[m * ldx + r] = src[e];
  }
}

// gW[n][k] += sum_m G[n][m] Xp[m][k] (n < Nn, k < Kk <= 128), gb[n] += sum_m G[n][m].
__device__ void outer_accum(const float* G, int Nn, const float* Xp, int ldx, int Kk,
                            float* __restrict__ gW, float* __restrict__ gb) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int n0 = 4 * warp; n0 < Nn; n0 += 4 * kWarps) {
    float acc[4][4], bs[4];
#pragma unroll
    for (int a = 0; a < 4; a++) {
      bs[a] = 0.f;
#pragma unroll
      for (int j = 0; j < 4; j++) acc[a][j] = 0.f;
    }
    for (int m = 0; m < kTM; m++) {
      float g[4], x[4];
#pragma unroll
      for (int a = 0; a < 4; a++) g[a] = (n0 + a < Nn) ? G[(n0 + a) * kTM + m] : 0.f;
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const int k = lane + 32 * j;
        x[j] = k < Kk ? Xp[m * ldx + k] : 0.f;
      }
#pragma unroll
      for (int a = 0; a < 4; a++) {
        bs[a] = __fadd_rn(bs[a], g[a]);
#pragma unroll
        for (int j = 0; j < 4; j++) acc[a][j] = __fmaf_rn(g[a], x[j], acc[a][j]);
      }
    }
#pragma unroll
    for (int a = 0; a < 4; a++) {
      if (n0 + a >= Nn) continue;
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const int k = lane + 32 * j;
        if (k < Kk) {
          float* o = gW + (size_t)(n0 + a) * Kk + k;
          *o = __fadd_rn(*o, acc[a][j]);
        }
      }
      if (gb && lane == 0) gb[n0 + a] = __fadd_rn(gb[n0 + a], bs[a]);
    }
  }
}

// Per-pixel NLL (nats) of the discretized logistic mixture with coupled
// means and its gradient with respect to the 10K network outputs (lane k
// handles component k); writes scale * dL/dP into DP[n][m].
__device__ float pixel_nll_grad(const float* P, int K, int r, int g, int b, float scale, float* DP,
                                int m, int NOp, int lane) {
  const unsigned full = 0xffffffffu;
  CompState cs;
  comp_init(P, K, lane, cs);
  const int v[3] = {r, g, b};
  float l = -INFINITY, dlm[3] = {0.f, 0.f, 0.f}, dll[3] = {0.f, 0.f, 0.f}, mm[3] = {0.f, 0.f, 0.f};
  if (lane < K) {
    l = cs.logpi;
    for (int c = 0; c < 3; c++) {
      const float mc = comp_mean(cs, c, r, g), inv = cs.inv[c];
      mm[c] = mc;
      l = __fadd_rn(l, log_bin_mass_f(mc, inv, cs.lme[c], v[c]));
      if (v[c] == 0) {
        const float a = __fmul_rn(__fsub_rn(edge_f(1), mc), inv);
        const float sa = 1.f / (1.f + expf(a));  // sigmoid(-a)
        dlm[c] = -inv * sa;
        dll[c] = -a * sa;
      } else if (v[c] == 255) {
        const float bb = __fmul_rn(__fsub_rn(edge_f(255), mc), inv);
        const float sb = 1.f / (1.f + expf(-bb));  // sigmoid(b)
        dlm[c] = inv * sb;
        dll[c] = bb * sb;
      } else {
        const float a = __fmul_rn(__fsub_rn(edge_f(v[c] + 1), mc), inv);
        const float bb = __fmul_rn(__fsub_rn(edge_f(v[c]), mc), inv);
        const float dd = __fmul_rn(__fdiv_rn(2.f, 255.f), inv);
        const float gk = 1.f / expm1f(dd);
        const float sa = 1.f / (1.f + expf(a)), sb = 1.f / (1.f + expf(-bb));
        dlm[c] = -inv * (sa - sb);
        dll[c] = -a * sa + bb * sb - gk * dd;
      }
    }
  }
  float mx = l;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(full, mx, o));
  float e = lane < K ? expf(__fsub_rn(l, mx)) : 0.f;
  float s = e;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s = __fadd_rn(s, __shfl_xor_sync(full, s, o));
  const float nll = -__fadd_rn(mx, logf(s));
  if (lane < K) {
    const float rho = e / s, pi = expf(cs.logpi);
    const float xr = __fdiv_rn((float)(2 * r - 255), 255.f);
    const float xg = __fdiv_rn((float)(2 * g - 255), 255.f);
    const float dmR = -rho * dlm[0], dmG = -rho * dlm[1], dmB = -rho * dlm[2];
    DP[(0 * K + lane) * kTM + m] = scale * (pi - rho);
    DP[(1 * K + lane) * kTM + m] = scale * dmR;
    DP[(2 * K + lane) * kTM + m] = scale * dmG;
    DP[(3 * K + lane) * kTM + m] = scale * dmB;
    for (int c = 0; c < 3; c++) {
      const float raw = P[4 * K + c * K + lane];
      DP[(4 * K + c * K + lane) * kTM + m] = raw > -7.f ? scale * (-rho * dll[c]) : 0.f;
    }
    const float al = cs.co[0], be = cs.co[1], ga = cs.co[2];
    DP[(7 * K + lane) * kTM + m] = scale * dmG * xr * (1.f - al * al);
    DP[(8 * K + lane) * kTM + m] = scale * dmB * xr * (1.f - be * be);
    DP[(9 * K + lane) * kTM + m] = scale * dmB * xg * (1.f - ga * ga);
  }
  (void)mm;
  (void)NOp;
  return nll;
}

// dparams == nullptr: dP = gradient of the batch's mean code length (bits
// per dimension); else dP = dparams [n_px][10K] (an upstream gradient of the
// network outputs, raster order of the batch) and no loss is computed.
__global__ void __launch_bounds__(kThreads, 1)
    loss_grad_kernel(Dims d, const float* __restrict__ w, const float* __restrict__ wt,
                     const uint8_t* __restrict__ batch, int N, int H, int W,
                     const float* __restrict__ dparams, float* __restrict__ part_g,
                     float* __restrict__ part_l, int n_w) {
  extern __shared__ __align__(16) float sm[];
  const TrainPlan pl = train_plan(d);
  float* X = sm + pl.X;
  float* A = sm + pl.A;
  float* Hp = sm + pl.Hp;
  float* P = sm + pl.P;
  float* DP = sm + pl.DP;
  float* T1 = sm + pl.T1;
  float* T2 = sm + pl.T2;
  float* XP = sm + pl.XP;
  float* zeros = sm + pl.zeros;
  float* red = sm + pl.red;
  PixSlot* slots = reinterpret_cast<PixSlot*>(sm + pl.end);
  const int C = d.C, F = d.F, R = d.R, K = d.K, NO = d.NO, ldP = d.ldP, h = d.h;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ldx = pl.ldx;
  float* gW = part_g + (size_t)blockIdx.x * n_w;
  for (int i = threadIdx.x; i < n_w; i += blockDim.x) gW[i] = 0.f;
  for (int i = threadIdx.x; i < (d.NOp > C ? d.NOp : C); i += blockDim.x) zeros[i] = 0.f;
  if (threadIdx.x < 32) red[threadIdx.x] = 0.f;
  // canonical offsets of the gradient / weights
  const size_t oW0 = 0, ob0 = (size_t)C * F, oblk = ob0 + C;
  const size_t blk = 2 * (size_t)C * C + 2 * C;
  const size_t oWH = oblk + (size_t)R * blk, obH = oWH + (size_t)NO * C;
  // packed transposed weights for the forward
  const float* W0T = wt;
  const float* b0 = W0T + (size_t)F * C;
  const float* WHT = b0 + C + (size_t)R * blk;
  const float* bH = WHT + (size_t)C * d.NOp;
  const long long HW = (long long)H * W, n_px = (long long)N * HW;
  const float scale = 1.f / (0.6931471805599453f * 3.f * (float)n_px);
  __syncthreads();
  const long long ntiles = (n_px + kTM - 1) / kTM;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    if (threadIdx.x < kTM) {
      const long long q = tile * kTM + threadIdx.x;
      PixSlot ps{-1, 0, 0, 0};
      if (q < n_px) {
        ps.unit = (int)(q / HW);
        const long long rr = q % HW;
        ps.i = (int)(rr / W);
        ps.j = (int)(rr % W);
      }
      slots[threadIdx.x] = ps;
    }
    __syncthreads();
    // gather (each image is one unit; zero outside it)
    const int ntap = 2 * h * (h + 1);
    for (int it = threadIdx.x; it < kTM * (d.Fp / 3 + 1); it += blockDim.x) {
      const int m = it % kTM, p = it / kTM;
      if (3 * p >= d.Fp) continue;
      const PixSlot s = slots[m];
      float v0 = 0.f, v1 = 0.f, v2 = 0.f;
      if (s.unit >= 0 && p < ntap) {
        int dy, dx;
        tap_offset(p, h, dy, dx);
        const int ii = s.i + dy, jj = s.j + dx;
        if (ii >= 0 && ii < H && jj >= 0 && jj < W) {
          const uint8_t* px = batch + ((long long)s.unit * HW + (long long)ii * W + jj) * 3;
          v0 = __fdiv_rn((float)(2 * px[0] - 255), 255.f);
          v1 = __fdiv_rn((float)(2 * px[1] - 255), 255.f);
          v2 = __fdiv_rn((float)(2 * px[2] - 255), 255.f);
        }
      }
      if (3 * p + 0 < d.Fp) X[(3 * p + 0) * kTM + m] = v0;
      if (3 * p + 1 < d.Fp) X[(3 * p + 1) * kTM + m] = v1;
      if (3 * p + 2 < d.Fp) X[(3 * p + 2) * kTM + m] = v2;
    }
    __syncthreads();
    // ---- forward ----
    gemm_dispatch<kTM>(GM_STORE, X, F, W0T, b0, C, A, 0);
    __syncthreads();
    for (int r = 0; r < R; r++) {
      const float* W1T = b0 + C + r * blk;
      const float* b1 = W1T + (size_t)C * C;
      const float* W2T = b1 + C;
      const float* b2 = W2T + (size_t)C * C;
      float* Ar = A + (size_t)r * C * kTM;
      float* An = Ar + (size_t)C * kTM;
      float* Hr = Hp + (size_t)r * C * kTM;
      for (int e = threadIdx.x; e < C * kTM; e += blockDim.x) {
        T1[e] = elu_f(Ar[e]);
        An[e] = Ar[e];
      }
      __syncthreads();
      gemm_dispatch<kTM>(GM_STORE, T1, C, W1T, b1, C, Hr, 0);
      __syncthreads();
      for (int e = threadIdx.x; e < C * kTM; e += blockDim.x) T2[e] = elu_f(Hr[e]);
      __syncthreads();
      gemm_dispatch<kTM>(GM_RESID, T2, C, W2T, b2, C, An, 0);
      __syncthreads();
    }
    float* AR = A + (size_t)R * C * kTM;
    for (int e = threadIdx.x; e < C * kTM; e += blockDim.x) T1[e] = elu_f(AR[e]);
    __syncthreads();
    gemm_dispatch<kTM>(GM_HEAD, T1, C, WHT, bH, d.NOp, P, ldP);
    __syncthreads();
    // ---- likelihood and its gradient ----
    for (int e = threadIdx.x; e < d.NOp * kTM; e += blockDim.x) DP[e] = 0.f;
    __syncthreads();
    for (int m = warp; m < kTM; m += kWarps) {
      const PixSlot s = slots[m];
      if (s.unit < 0) continue;
      if (dparams) {
        const long long q = tile * kTM + m;
        for (int k = lane; k < NO; k += 32) DP[k * kTM + m] = dparams[q * NO + k];
        continue;
      }
      const uint8_t* px = batch + ((long long)s.unit * HW + (long long)s.i * W + s.j) * 3;
      const float nll = pixel_nll_grad(P + (size_t)m * ldP, K, px[0], px[1], px[2], scale, DP, m,
                                       d.NOp, lane);
      if (lane == 0) red[warp] = __fadd_rn(red[warp], nll);
    }
    __syncthreads();
    // ---- adjoint ----
    to_pixel_major(T1, C, XP, ldx);  // ELU(a_R)
    __syncthreads();
    outer_accum(DP, NO, XP, ldx, C, gW + oWH, gW + obH);
    // dELU(a_R) = WH^T dP
    gemm_dispatch<kTM>(GM_STORE, DP, NO, w + oWH, zeros, C, T2, 0);
    __syncthreads();
    for (int e = threadIdx.x; e < C * kTM; e += blockDim.x)
      T2[e] = __fmul_rn(T2[e], elu_d(AR[e]));
    __syncthreads();
    for (int r = R - 1; r >= 0; r--) {
      const size_t oW1 = oblk + r * blk, ob1 = oW1 + (size_t)C * C;
      const size_t oW2 = ob1 + C, ob2 = oW2 + (size_t)C * C;
      float* Ar = A + (size_t)r * C * kTM;
      float* Hr = Hp + (size_t)r * C * kTM;
      for (int e = threadIdx.x; e < C * kTM; e += blockDim.x) T1[e] = elu_f(Hr[e]);
      __syncthreads();
      to_pixel_major(T1, C, XP, ldx);
      __syncthreads();
      outer_accum(T2, C, XP, ldx, C, gW + oW2, gW + ob2);
      gemm_dispatch<kTM>(GM_STORE, T2, C, w + oW2, zeros, C, P, 0);  // dv = W2^T da
      __syncthreads();
      for (int e = threadIdx.x; e < C * kTM; e += blockDim.x) {
        P[e] = __fmul_rn(P[e], elu_d(Hr[e]));  // d hidden pre-activation
        T1[e] = elu_f(Ar[e]);
      }
      __syncthreads();
      to_pixel_major(T1, C, XP, ldx);
      __syncthreads();
      outer_accum(P, C, XP, ldx, C, gW + oW1, gW + ob1);
      gemm_dispatch<kTM>(GM_STORE, P, C, w + oW1, zeros, C, T1, 0);  // du = W1^T dh
      __syncthreads();
      for (int e = threadIdx.x; e < C * kTM; e += blockDim.x)
        T2[e] = __fadd_rn(T2[e], __fmul_rn(T1[e], elu_d(Ar[e])));
      __syncthreads();
    }
    to_pixel_major(X, F, XP, ldx);
    __syncthreads();
    outer_accum(T2, C, XP, ldx, F, gW + oW0, gW + ob0);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < kWarps; i++) t = __fadd_rn(t, red[i]);
    part_l[blockIdx.x] = t;
  }
}

__global__ void reduce_grad_kernel(const float* __restrict__ part_g, const float* __restrict__ part_l,
                                   int nblk, int n_w, int ldw, float inv_dims,
                                   float* __restrict__ grad, float* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_w) {
    float s = 0.f;
    for (int b = 0; b < nblk; b++) s = __fadd_rn(s, part_g[(size_t)b * ldw + i]);
    grad[i] = s;
  }
  if (i == 0 && part_l && loss) {
    float s = 0.f;
    for (int b = 0; b < nblk; b++) s = __fadd_rn(s, part_l[b]);
    *loss = s * inv_dims;
  }
}

cudaError_t launch_reduce_grad(const float* part_g, const float* part_l, int nblk, int n_w, int ldw,
                               long long n_px, float* grad, float* loss, cudaStream_t s) {
  const float inv_dims = 1.f / (0.6931471805599453f * 3.f * (float)n_px);
  reduce_grad_kernel<<<(n_w + 255) / 256, 256, 0, s>>>(part_g, part_l, nblk, n_w, ldw, inv_dims,
                                                      grad, loss);
  return cudaGetLastError();
}

bool simt_train_fits(const Dims& d) { return train_smem_bytes(d) <= 227 * 1024; }

static int train_grid(long long n_px, int sm_count) {
  long long t = (n_px + kTM - 1) / kTM;
  return (int)(t < sm_count ? (t < 1 ? 1 : t) : sm_count);
}

size_t train_ws_bytes(const Dims& d, long long n_px, int sm_count) {
  const size_t nw = (size_t)d.C * d.F + d.C + (size_t)d.R * (2 * d.C * d.C + 2 * d.C) +
                    (size_t)d.NO * d.C + d.NO;
  const int g = train_grid(n_px, sm_count);
  return ((size_t)g * nw + g + 64) * 4;
}

cudaError_t launch_loss_grad(const Dims& d, const float* w, const float* wt, const uint8_t* batch,
                             int N, int H, int W, const float* dparams, float* loss, float* grad,
                             void* ws, int sm_count, cudaStream_t s) {
  const int n_w = (int)((size_t)d.C * d.F + d.C + (size_t)d.R * (2 * d.C * d.C + 2 * d.C) +
                        (size_t)d.NO * d.C + d.NO);
  const long long n_px = (long long)N * H * W;
  const int g = train_grid(n_px, sm_count);
  const size_t smem = train_smem_bytes(d);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(loss_grad_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  float* part_g = reinterpret_cast<float*>(ws);
  float* part_l = part_g + (size_t)g * n_w;
  loss_grad_kernel<<<g, kThreads, smem, s>>>(d, w, wt, batch, N, H, W, dparams, part_g, part_l,
                                              n_w);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_reduce_grad(part_g, dparams ? nullptr : part_l, g, n_w, n_w, n_px, grad, loss, s);
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

cudaError_t launch_adam(float* w, const float* g, float* m, float* v, int n, float lr, float b1,
                        float b2, float eps, long long t, cudaStream_t s) {
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  adam_kernel<<<(n + 255) / 256, 256, 0, s>>>(w, g, m, v, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace nlc
