// Encoder stage 1 (every pixel's frequency tables, all pixels in parallel,
// with the decoder's own device code) and the forward entry point.
#include "nlc_tile.cuh"

namespace nlc {

// ---------------------------------------------------------------------
// Encoder, stage 1: the (start, freq) of every symbol, all pixels in
// parallel (the decoder's tables, computed by the same device code).
// ---------------------------------------------------------------------
template <int PREC>
__global__ void __launch_bounds__(kThreads, 1)
    enc_tables_kernel(DeviceModel m, const Unit* __restrict__ units, int n_units, long long n_px,
                      uint32_t* __restrict__ stage) {
  extern __shared__ __align__(128) unsigned char smem[];
  TileSmem t = carve(m.d, smem, 0);
  if constexpr (PREC == PREC_BF16) tc_setup(t.tc);
  load_weights<PREC>(m, t);
  __syncthreads();
  constexpr int MT = tile_size<PREC>();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int K = m.d.K;
  const long long ntiles = (n_px + MT - 1) / MT;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    for (int s = threadIdx.x; s < MT; s += blockDim.x) {
      long long q = tile * MT + s;
      PixSlot ps{-1, 0, 0, 0};
      if (q < n_px) {
        int u = find_unit_px(units, n_units, q);
        const Unit U = units[u];
        long long r = q - U.px_base;
        ps.unit = u;
        ps.i = (int)(r / U.Wu);
        ps.j = (int)(r % U.Wu);
      }
      t.slots[s] = ps;
    }
    __syncthreads();
    tile_network<PREC, false>(m, units, t, (int)min((long long)MT, n_px - tile * MT));
    // two pixels per warp, one per 16-lane coding group (as in the decoder)
    const int half = lane >> 4, gl = lane & (kGW - 1);
    for (int j = 0; 2 * warp + kGroups * j < MT; j++) {
      const int s = 2 * warp + half + kGroups * j;
      const bool valid = t.slots[s].unit >= 0;
      if (!__any_sync(0xffffffffu, valid)) break;
      const int se = valid ? s : (s ^ 1);  // an idle group shadows its neighbour
      const PixSlot ps = t.slots[se];
      const Unit U = units[ps.unit];
      const uint8_t* px = U.img + ((long long)(U.y0 + ps.i) * U.img_W + (U.x0 + ps.j)) * 3;
      const int v[3] = {px[0], px[1], px[2]};
      const long long q = tile * MT + s;
      WarpScratch& ws = t.ws[2 * warp + half];
      CompState cs;
      comp_init<kGW>(tile_params(t, m.d, se), K, gl, cs);
      for (int ch = 0; ch < 3; ch++) {
        int nact;
        const float mloc = channel_setup<kGW>(cs, K, ch, v[0], v[1], gl, ws, nact);
        uint32_t c0, c1;
        cdf_pair<kGW>(ws, v[ch], gl, c0, c1);
        if (gl == 0 && valid) stage[3 * q + ch] = c0 | ((c1 - c0) << 16);
        if (ch < 2) comp_observe(cs, K, ch, mloc, v[ch], gl);
        __syncwarp();
      }
    }
    __syncthreads();
  }
  if constexpr (PREC == PREC_BF16) tc_teardown(t.tc);
}

// Encoder, stage 2: one thread per stream, reverse order.

cudaError_t launch_enc_tables(const DeviceModel& m, const CodecBufs& b, int sm_count,
                              cudaStream_t s) {
  const size_t smem = tile_smem_bytes(m.d, 0);
  const bool tc = m.d.prec == PREC_BF16;
  const void* fn =
      tc ? (const void*)enc_tables_kernel<PREC_BF16> : (const void*)enc_tables_kernel<PREC_FP32>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int MT = tc ? kTcM : kMT;
  const int grid = grid_for((b.n_px + MT - 1) / MT, 1, sm_count);
  if (tc)
    enc_tables_kernel<PREC_BF16><<<grid, kThreads, smem, s>>>(m, b.units, b.n_units, b.n_px, b.stage);
  else
    enc_tables_kernel<PREC_FP32><<<grid, kThreads, smem, s>>>(m, b.units, b.n_units, b.n_px, b.stage);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------
// Forward (network outputs and/or model code length of every pixel).
// ---------------------------------------------------------------------
template <int PREC>
__global__ void __launch_bounds__(kThreads, 1)
    forward_kernel(DeviceModel m, const Unit* __restrict__ units, int n_units, long long n_px,
                   float* __restrict__ params, float* __restrict__ bits) {
  extern __shared__ __align__(128) unsigned char smem[];
  TileSmem t = carve(m.d, smem, 0);
  if constexpr (PREC == PREC_BF16) tc_setup(t.tc);
  load_weights<PREC>(m, t);
  __syncthreads();
  constexpr int MT = tile_size<PREC>();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int K = m.d.K, NO = m.d.NO;
  const long long ntiles = (n_px + MT - 1) / MT;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    for (int s = threadIdx.x; s < MT; s += blockDim.x) {
      long long q = tile * MT + s;
      PixSlot ps{-1, 0, 0, 0};
      if (q < n_px) {
        int u = find_unit_px(units, n_units, q);
        const Unit U = units[u];
        long long r = q - U.px_base;
        ps.unit = u;
        ps.i = (int)(r / U.Wu);
        ps.j = (int)(r % U.Wu);
      }
      t.slots[s] = ps;
    }
    __syncthreads();
    tile_network<PREC, false>(m, units, t, (int)min((long long)MT, n_px - tile * MT));
    for (int s = warp; s < MT; s += kWarps) {
      const PixSlot ps = t.slots[s];
      if (ps.unit < 0) continue;
      const Unit U = units[ps.unit];
      // outputs in image raster order
      const long long q = U.img_px_base + (long long)(U.y0 + ps.i) * U.img_W + (U.x0 + ps.j);
      const float* P = tile_params(t, m.d, s);
      if (params)
        for (int k = lane; k < NO; k += 32) params[q * NO + k] = P[k];
      if (bits) {
        const uint8_t* px = U.img + ((long long)(U.y0 + ps.i) * U.img_W + (U.x0 + ps.j)) * 3;
        const int v[3] = {px[0], px[1], px[2]};
        CompState cs;
        comp_init(P, K, lane, cs);
        float l = -INFINITY;
        if (lane < K) {
          l = cs.logpi;
          for (int ch = 0; ch < 3; ch++)
            l = __fadd_rn(l, log_bin_mass_f(comp_mean(cs, ch, v[0], v[1]), cs.inv[ch],
                                             cs.lme[ch], v[ch]));
        }
        float mx = l;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        float e = lane < K ? expf(__fsub_rn(l, mx)) : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e = __fadd_rn(e, __shfl_xor_sync(0xffffffffu, e, o));
        if (lane == 0) bits[q] = -__fadd_rn(mx, logf(e)) * 1.4426950408889634f;
      }
    }
    __syncthreads();
  }
  if constexpr (PREC == PREC_BF16) tc_teardown(t.tc);
}

cudaError_t launch_forward(const DeviceModel& m, const CodecBufs& b, float* params, float* bits,
                           int sm_count, cudaStream_t s) {
  if (b.n_px == 0) return cudaSuccess;
  const size_t smem = tile_smem_bytes(m.d, 0);
  const bool tc = m.d.prec == PREC_BF16;
  const void* fn = tc ? (const void*)forward_kernel<PREC_BF16> : (const void*)forward_kernel<PREC_FP32>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int MT = tc ? kTcM : kMT;
  const int grid = grid_for((b.n_px + MT - 1) / MT, 1, sm_count);
  if (tc)
    forward_kernel<PREC_BF16><<<grid, kThreads, smem, s>>>(m, b.units, b.n_units, b.n_px, params, bits);
  else
    forward_kernel<PREC_FP32><<<grid, kThreads, smem, s>>>(m, b.units, b.n_units, b.n_px, params, bits);
  return cudaGetLastError();
}


}  // namespace nlc
