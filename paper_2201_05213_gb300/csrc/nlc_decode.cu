// The wavefront decoder (Algorithm 1, Section 3) as one persistent
// cooperative kernel, and its launcher.
#include "nlc_tile.cuh"

namespace nlc {

// ---------------------------------------------------------------------
// Decoder: persistent cooperative kernel.  Step t decodes, for every unit,
// the pixels of its front (wavefront: j = tau - (h+1) i, Section 3; raster:
// one pixel).  The step's pixels are split evenly across the CTAs; each CTA
// runs gather -> network -> per-pixel CDF + rANS for its share, then all
// CTAs meet at a grid barrier before step t+1.
// ---------------------------------------------------------------------
struct DecodeArgs {
  DeviceModel m;
  const Unit* units;
  int n_units;
  int layout, sched, T;
  const uint8_t* in;
  uint32_t* st_x;
  unsigned long long* st_pos;
  const unsigned long long* st_end;
  unsigned* bar;
  int* status;
  unsigned long long* prof;  // optional per-phase cycle counters
};

// Slot of the warp's l-th pixel when coding groups have GW lanes
// (32 / GW groups per warp, group g of warp w takes slots g + 32/GW (w + 8 j)).
template <int GW>
__device__ __forceinline__ int group_slot(int warp, int l) {
  constexpr int gpw = 32 / GW;
  return gpw * warp + (l % gpw) + kWarps * gpw * (l / gpw);
}

// Codes the tile's pixels: per pixel, the R, G|r, B|r,g tables and one rANS
// symbol each.  pd holds (in lane l) the prefetched stream state of the
// warp's l-th pixel.
template <int GW>
__device__ __noinline__ void code_tile(const DecodeArgs& a, const TileSmem& t, int n,
                                       const GroupRansDec& pd) {
  constexpr int gpw = 32 / GW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / GW, gl = lane % GW;
  const int K = a.m.d.K, ldP = a.m.d.ldP;
  // sub-stage cycles of thread 0: mixture set-up, tables, rANS, posterior
  const bool prof = a.prof != nullptr && threadIdx.x == 0;
  long long s_init = 0, s_tab = 0, s_dec = 0, s_obs = 0, s_px = 0, c0 = 0, c1 = 0;
  for (int j = 0; gpw * warp + kWarps * gpw * j < n; j++) {
    const int s = gpw * warp + grp + kWarps * gpw * j;
    const bool valid = s < n;
    const int se = valid ? s : s - 1;  // an idle group shadows its neighbour
    const int src = gpw * j + grp;
    GroupRansDec dec;
    dec.x = __shfl_sync(0xffffffffu, pd.x, src);
    dec.pos = __shfl_sync(0xffffffffu, pd.pos, src);
    dec.end = __shfl_sync(0xffffffffu, pd.end, src);
    dec.lo = __shfl_sync(0xffffffffu, pd.lo, src);
    dec.hi = __shfl_sync(0xffffffffu, pd.hi, src);
    dec.used = 0;
    dec.bad = false;
    const PixSlot ps = t.slots[se];
    const Unit U = a.units[ps.unit];
    const int sid = ps.aux;
    WarpScratch& ws = t.ws[gpw * warp + grp];
    CompState cs;
    if (prof) c0 = clock64();
    comp_init<GW>(t.U0 + (size_t)se * ldP, K, gl, cs);
    if (prof) { c1 = clock64(); s_init += c1 - c0; c0 = c1; s_px++; }
    int v[3] = {0, 0, 0};
    for (int ch = 0; ch < 3; ch++) {
      int nact;
      const float mloc = channel_setup<GW>(cs, K, ch, v[0], v[1], gl, ws, nact);
      if (prof) { c1 = clock64(); s_init += c1 - c0; c0 = c1; }
      const uint32_t slot = dec.x & 0xFFFFu;
      uint32_t lo, hi;
      v[ch] = cdf_search<GW>(ws, nact, slot, gl, lo, hi);
      if (prof) { c1 = clock64(); s_tab += c1 - c0; c0 = c1; }
      dec.advance(slot, lo, hi);
      if (prof) { c1 = clock64(); s_dec += c1 - c0; c0 = c1; }
      if (ch < 2) comp_observe(cs, K, ch, mloc, v[ch], gl);
      __syncwarp();
      if (prof) { c1 = clock64(); s_obs += c1 - c0; c0 = c1; }
    }
    if (gl == 0 && valid) {
      uint8_t* px = U.img + ((long long)(U.y0 + ps.i) * U.img_W + (U.x0 + ps.j)) * 3;
      px[0] = (uint8_t)v[0];
      px[1] = (uint8_t)v[1];
      px[2] = (uint8_t)v[2];
      const unsigned long long np = dec.pos + (unsigned long long)dec.used;
      a.st_x[sid] = dec.x;
      a.st_pos[sid] = np;
      const bool last = a.layout == 1 ? (ps.j == U.Wu - 1) : (ps.i == U.Hu - 1 && ps.j == U.Wu - 1);
      if (dec.bad || (last && (dec.x != kRansL || np != dec.end))) set_status(a.status, ST_CORRUPT);
    }
  }
  if (prof) {
    atomicAdd(a.prof + 8, (unsigned long long)s_init);
    atomicAdd(a.prof + 9, (unsigned long long)s_tab);
    atomicAdd(a.prof + 10, (unsigned long long)s_dec);
    atomicAdd(a.prof + 11, (unsigned long long)s_obs);
    atomicAdd(a.prof + 12, (unsigned long long)s_px);
  }
}

template <int PREC>
__global__ void __launch_bounds__(kThreads, 1) decode_kernel(DecodeArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Dims& d = a.m.d;
  TileSmem t = carve(d, smem, a.n_units);
  if constexpr (PREC == PREC_BF16) tc_setup(t.tc);
  load_weights<PREC>(a.m, t);
  if (threadIdx.x == 0) t.flag[0] = 0;
  __syncthreads();
  constexpr int MT = tile_size<PREC>();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int h = d.h;
  unsigned my_gen = 0;
  const unsigned G = gridDim.x;
  // phase cycles of thread 0: front scan, slot fill, gather + network,
  // per-pixel coding, grid barrier
  const bool prof = a.prof != nullptr && threadIdx.x == 0;
  long long ph0 = 0, ph1 = 0, ph2 = 0, ph3 = 0, ph4 = 0, tiles = 0, tc = 0, tn = 0;
  for (int step = 0; step < a.T; step++) {
    if (prof) tc = clock64();
    const int F = front_scan(a.units, a.n_units, step, h, a.sched, t.pre, t.sh);
    if (prof) { tn = clock64(); ph0 += tn - tc; tc = tn; }
    const long long lo = (long long)F * blockIdx.x / G, hi = (long long)F * (blockIdx.x + 1) / G;
    for (long long base = lo; base < hi; base += MT) {
      const int n = (int)min((long long)MT, hi - base);
      for (int s = threadIdx.x; s < MT; s += blockDim.x) {
        PixSlot ps{-1, 0, 0, 0};
        if (s < n) {
          const int q = (int)(base + s);
          int lo2 = 0, hi2 = a.n_units - 1;  // last u with pre[u] <= q
          while (lo2 < hi2) {
            int mid = (lo2 + hi2 + 1) >> 1;
            if (t.pre[mid] <= q) lo2 = mid; else hi2 = mid - 1;
          }
          const Unit U = a.units[lo2];
          const Front fr = unit_front(U, step, h, a.sched);
          ps.unit = lo2;
          ps.i = fr.i_lo + (q - t.pre[lo2]);
          ps.j = front_col(U, step, ps.i, h, a.sched);
          ps.aux = U.stream_base + (a.layout == 1 ? ps.i : 0);
        }
        t.slots[s] = ps;
      }
      __syncthreads();
      // A CTA with at most one pixel per warp codes with whole warps (lower
      // latency per pixel); otherwise two pixels per warp.  Both give the
      // same tables (see channel_table).  Lane l of warp w fetches the rANS
      // state and next 8 bytes of the warp's l-th pixel ahead of the network.
      const bool wide = n <= kWarps;
      GroupRansDec pd;
      pd.x = 0;
      pd.pos = pd.end = 0;
      pd.lo = pd.hi = 0;
      {
        const int sl = wide ? group_slot<32>(warp, lane) : group_slot<kGW>(warp, lane);
        if (sl < n) {
          const int sid = t.slots[sl].aux;
          pd.x = ld_cg_u32(a.st_x + sid);
          pd.pos = ld_cg_u64(a.st_pos + sid);
          pd.end = a.st_end[sid];
          pd.load_bytes(a.in);
        }
      }
      if (prof) { tn = clock64(); ph1 += tn - tc; tc = tn; tiles++; }
      tile_network<PREC, true>(a.m, a.units, t, n);
      if (prof) { tn = clock64(); ph2 += tn - tc; tc = tn; }
      if (wide) code_tile<32>(a, t, n, pd);
      else code_tile<kGW>(a, t, n, pd);
      __syncthreads();
      if (prof) { tn = clock64(); ph3 += tn - tc; tc = tn; }
    }
    if (G > 1) {
      if (!grid_barrier(a.bar, a.bar + 1, G, my_gen, a.status, t.flag)) break;
    } else {
      __syncthreads();
    }
    if (prof) ph4 += clock64() - tc;
  }
  if (prof) {
    atomicAdd(a.prof + 0, (unsigned long long)ph0);
    atomicAdd(a.prof + 1, (unsigned long long)ph1);
    atomicAdd(a.prof + 2, (unsigned long long)ph2);
    atomicAdd(a.prof + 3, (unsigned long long)ph3);
    atomicAdd(a.prof + 4, (unsigned long long)ph4);
    atomicAdd(a.prof + 5, (unsigned long long)tiles);
    atomicAdd(a.prof + 6, 1ull);
    if (blockIdx.x == 0) atomicAdd(a.prof + 7, (unsigned long long)a.T);
  }
  if constexpr (PREC == PREC_BF16) tc_teardown(t.tc);
}

size_t decode_smem_bytes(const Dims& d, int n_units) { return tile_smem_bytes(d, n_units); }

static const void* decode_fn(int prec) {
  return prec == PREC_BF16 ? (const void*)decode_kernel<PREC_BF16>
                           : (const void*)decode_kernel<PREC_FP32>;
}

int decode_max_grid(const DeviceModel& m, int n_units, int sm_count) {
  const size_t smem = decode_smem_bytes(m.d, n_units);
  const void* fn = decode_fn(m.d.prec);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kThreads, smem) != cudaSuccess)
    return 0;
  return per * sm_count;
}

cudaError_t launch_decode(const DeviceModel& m, const CodecBufs& b, const uint8_t* in,
                          const unsigned long long* d_offsets, int layout, int patch, int sched,
                          int T, int grid, cudaStream_t s) {
  cudaError_t e;
  if (b.n_images == 0) return cudaSuccess;
  if ((e = launch_parse(m, b, in, d_offsets, layout, patch, s)) != cudaSuccess) return e;
  if (b.n_units == 0) return cudaSuccess;
  if ((e = cudaMemsetAsync(b.bar, 0, 2 * sizeof(unsigned), s)) != cudaSuccess) return e;
  DecodeArgs a;
  a.m = m;
  a.units = b.units;
  a.n_units = b.n_units;
  a.layout = layout;
  a.sched = sched;
  a.T = T;
  a.in = in;
  a.st_x = b.st_x;
  a.st_pos = b.st_pos;
  a.st_end = b.st_end;
  a.bar = b.bar;
  a.status = b.status;
  a.prof = b.prof;
  const size_t smem = decode_smem_bytes(m.d, b.n_units);
  const void* fn = decode_fn(m.d.prec);
  if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
      cudaSuccess)
    return e;
  void* args[] = {&a};
  if (grid > 1) return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kThreads), args, smem, s);
  return cudaLaunchKernel(fn, dim3(1), dim3(kThreads), args, smem, s);
}

}  // namespace nlc
