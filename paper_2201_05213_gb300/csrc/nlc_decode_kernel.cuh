// The wavefront decoder's device code (Algorithm 1, Section 3): the
// persistent cooperative kernel and its coding functions.  Included by
// nlc_decode.cu (the launchers and the plain build) and nlc_decode_prof.cu
// (the instrumented build behind nlc_decode_profile), so that each
// compilation unit holds one build: in one unit together, ptxas gave the
// plain build's coding function and step loop more spills.
#pragma once
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
  StreamRec* st;
  unsigned* bar;
  int* status;
  unsigned long long* prof;  // optional per-phase cycle counters
  unsigned long long* times;  // optional: [0] start, [t + 1] end of step t (ns)
  long long n_times;
  unsigned long long seed;    // sampler only
  uint8_t* ring;              // sheared wavefront decoder: the units' sheared rings
  unsigned spin_limit;        // polls of the grid barrier before a timeout
  unsigned mma_limit;         // polls of an MMA completion before a timeout
};

// Threads of the decoder's CTA: the BF16 pipeline runs 16 warps (32 coding
// groups of 16 lanes); the FP32 SIMT network is written for 256 threads.
template <int PREC>
__host__ __device__ constexpr int decode_threads() { return PREC == PREC_BF16 ? 512 : kThreads; }

// Slot of the warp's l-th pixel when coding groups have GW lanes and the
// CTA has NW warps (32 / GW groups per warp, group g of warp w takes slots
// g + 32/GW (w + NW j)).
template <int GW, int NW>
__device__ __forceinline__ int group_slot(int warp, int l) {
  constexpr int gpw = 32 / GW;
  return gpw * warp + (l % gpw) + NW * gpw * (l / gpw);
}

// Codes the tile's pixels: per pixel, the R, G|r, B|r,g symbols.  The
// pixels' stream records are in t.rec (visible to the warp), their windows
// are being copied to t.win by the warp's lanes.  With pc non-null, thread 0
// accumulates its sub-stage cycles in pc[8..12].
// Stores a decoded pixel in its unit's ring row at the byte offset rofs
// that the tile's schedule computed (slots tau mod 16 and tau mod 16 + 16 of
// its sheared column tau).
__device__ __forceinline__ void ring_put(const DecodeArgs& a, int rofs, const int (&v)[3]) {
  uint8_t* r = a.ring + rofs;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    r[c] = (uint8_t)v[c];
    r[48 + c] = (uint8_t)v[c];
  }
}

template <int GW, int NW, bool SHEAR, bool PROF>
__device__ __noinline__ void code_tile(const DecodeArgs& a, const TileSmem& t, int n,
                                       long long* pc) {
  constexpr int gpw = 32 / GW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / GW, gl = lane % GW;
  const int K = a.m.d.K;
  const bool pr = PROF && pc != nullptr && threadIdx.x == 0;
  long long ck = 0;
  auto tick = [&](int slot) {
    if (pr) {
      const long long n_ = clock64();
      pc[slot] += n_ - ck;
      ck = n_;
    }
  };
  for (int j = 0; gpw * warp + NW * gpw * j < n; j++) {
    const int s = gpw * warp + grp + NW * gpw * j;
    const bool valid = s < n;
    const int se = valid ? s : s - 1;  // an idle group shadows its neighbour
    GroupRansDec dec;
    {
      const uint4 q = *reinterpret_cast<const uint4*>(t.rec + se);
      const ulonglong2 pe = *reinterpret_cast<const ulonglong2*>(&t.rec[se].pos);
      dec.x = q.x;
      dec.lo = q.y;
      dec.hi = q.z;
      dec.set_avail(pe.x, pe.y);  // the positions are read again when the pixel is done
    }
    dec.w2 = dec.w3 = 0;
    dec.used = 0;
    dec.bad = false;
    const PixSlot ps = t.slots[se];
    WarpScratch& ws = t.ws[gpw * warp + grp];
    CompState cs;
    if (pr) {
      ck = clock64();
      pc[12] += 1;
    }
    comp_init<GW>(tile_params(t, a.m.d, SHEAR ? t.prow[se] : se), K, gl, cs);
    int v[3] = {0, 0, 0};
    for (int ch = 0; ch < 3; ch++) {
      int nact;
      const float mloc = channel_setup<GW>(cs, K, ch, v[0], v[1], gl, ws, nact);
      tick(8);
      const uint32_t slot = dec.x & 0xFFFFu;
      uint32_t lo, hi;
      v[ch] = cdf_search<GW>(ws, nact, slot, gl, lo, hi);
      tick(9);
      dec.advance(slot, lo, hi);
      tick(10);
      if (ch < 2) comp_observe(cs, K, ch, mloc, v[ch], gl);
      __syncwarp();
      tick(11);
    }
    cp_async_wait_all();  // the window copies of the warp's lanes
    __syncwarp();
    if (gl == 0 && valid) {
      const ulonglong2 pe = *reinterpret_cast<const ulonglong2*>(&t.rec[s].pos);
      dec.set_window(t.win + 4 * s, pe.x);
      const Unit U = a.units[ps.unit];
      uint8_t* px = U.img + ((long long)(U.y0 + ps.i) * U.img_W + (U.x0 + ps.j)) * 3;
      px[0] = (uint8_t)v[0];
      px[1] = (uint8_t)v[1];
      px[2] = (uint8_t)v[2];
      if (SHEAR) ring_put(a, t.rofs[s], v);
      const int sid = ps.aux;
      const unsigned long long np = pe.x + (unsigned long long)dec.used;
      uint32_t n0, n1;
      dec.next_bytes(n0, n1);
      StreamRec* r = a.st + sid;
      *reinterpret_cast<uint4*>(r) = make_uint4(dec.x, n0, n1, 0u);
      r->pos = np;
      const bool last = a.layout == 1 ? (ps.j == U.Wu - 1) : (ps.i == U.Hu - 1 && ps.j == U.Wu - 1);
      if (dec.bad || (last && (dec.x != kRansL || np != pe.y))) set_status(a.status, ST_CORRUPT);
    }
  }
}

// Draws the tile's pixels from the model (Section 5: the parallel schedules
// apply to sampling from a local autoregressive model): the symbol of each
// channel is the one whose quantised interval [cum_v, cum_{v+1}) holds a
// uniform 16-bit value from the counter-based generator (inverse-CDF
// sampling of the coder's own table), found by the decoder's search.
template <int GW, int NW, bool SHEAR>
__device__ __noinline__ void sample_tile(const DecodeArgs& a, const TileSmem& t, int n) {
  constexpr int gpw = 32 / GW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / GW, gl = lane % GW;
  const int K = a.m.d.K;
  for (int j = 0; gpw * warp + NW * gpw * j < n; j++) {
    const int s = gpw * warp + grp + NW * gpw * j;
    const bool valid = s < n;
    const int se = valid ? s : s - 1;  // an idle group shadows its neighbour
    const PixSlot ps = t.slots[se];
    const Unit U = a.units[ps.unit];
    const int y = U.y0 + ps.i, x = U.x0 + ps.j;
    WarpScratch& ws = t.ws[gpw * warp + grp];
    CompState cs;
    comp_init<GW>(tile_params(t, a.m.d, SHEAR ? t.prow[se] : se), K, gl, cs);
    int v[3] = {0, 0, 0};
    for (int ch = 0; ch < 3; ch++) {
      int nact;
      const float mloc = channel_setup<GW>(cs, K, ch, v[0], v[1], gl, ws, nact);
      const uint32_t u = sample_u16(a.seed, U.image, y, x, ch);
      uint32_t lo, hi;
      v[ch] = cdf_search<GW>(ws, nact, u, gl, lo, hi);
      if (ch < 2) comp_observe(cs, K, ch, mloc, v[ch], gl);
      __syncwarp();
    }
    if (gl == 0 && valid) {
      uint8_t* px = U.img + ((long long)y * U.img_W + x) * 3;
      px[0] = (uint8_t)v[0];
      px[1] = (uint8_t)v[1];
      px[2] = (uint8_t)v[2];
      if (SHEAR) ring_put(a, t.rofs[s], v);
    }
  }
}

// SHEAR: the sheared model's wavefront decoder (Section 3.1): decoded pixels
// also go to per-unit sheared rings, and each tile's context is one window
// tile of (unit, row) rows read from the rings, every unit's piece of the
// front preceded by h halo rows, with the first layer's MMAs reading the
// window rows of output row m at rows m .. m + h.
// PROF: the instrumented build behind nlc_decode_profile.  The cycle
// counters' state, live through the whole step loop even while profiling is
// off, cost the uninstrumented decoder 7 % (register spills), so only
// launches with a counter buffer run this instantiation.
template <int PREC, bool SAMPLE, bool SHEAR, bool PROF>
__global__ void __launch_bounds__(decode_threads<PREC>(), 1) decode_kernel(DecodeArgs a) {
  constexpr int NT = decode_threads<PREC>(), NW = NT / 32;
  extern __shared__ __align__(128) unsigned char smem[];
  const Dims& d = a.m.d;
  TileSmem t = carve(d, smem, a.n_units, NT / kGW, true);
  if constexpr (PREC == PREC_BF16) {
    tc_setup(t.tc);
    t.tc.mma_limit = a.mma_limit;
  }
  load_weights<PREC>(a.m, t);
  if (threadIdx.x == 0) t.flag[0] = 0;
  if (threadIdx.x < 16) t.pc[threadIdx.x] = 0;
  __syncthreads();
  // step end times: CTA 0 stamps each step when the grid barrier after it
  // releases (every CTA has finished it); every CTA stamps the last step's end
  const bool stamp = a.times != nullptr && threadIdx.x == 0;
  if (stamp && blockIdx.x == 0 && a.n_times > 0) a.times[0] = global_ns();
  constexpr int MT = tile_size<PREC>();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int h = d.h;
  const unsigned G = gridDim.x;
  // phase cycles of thread 0 (shared-memory accumulators): [0] front scan,
  // [1] slot fill, [2] gather + network, [3] per-pixel coding, [4] grid
  // barrier, [5] tiles
  long long* pc = PROF && a.prof != nullptr ? t.pc : nullptr;
  const bool pr = pc != nullptr && threadIdx.x == 0;
  long long ck = 0;
  auto tick = [&](int slot) {
    if (pr) {
      const long long n_ = clock64();
      pc[slot] += n_ - ck;
      ck = n_;
    }
  };
  // slots of the tile of n pixels starting at front position base of step
  // (by the first nt threads)
  auto fill_slots = [&](int step, long long base, int n, int nt) {
    for (int s = threadIdx.x; s < MT; s += nt) {
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
        if constexpr (SHEAR)  // ring bytes of the pixel's sheared column j + (h+1) i
          t.rofs[s] = kRingRowBytes * (U.ring_row + ps.i) + 3 * ((ps.j + (h + 1) * ps.i) & 15);
      }
      t.slots[s] = ps;
    }
  };
  // Sheared tile of at most nmax pixels from front position base: the
  // pixels' slots, their output rows prow (pixel s of the tile's k-th unit
  // piece at s + h k: each piece is preceded by h halo window rows), the
  // window rows' (unit, unit row), and t.flag[1..3] = the tile's pixels,
  // output rows and window rows (the output rows stay below MT).
  auto fill_slots_shear = [&](int step, long long base, int nmax, int nt) {
    fill_slots(step, base, nmax, nt);
    part_sync(nt);
    if (threadIdx.x < MT) {  // warps 0 .. MT/32 - 1
      const int s = threadIdx.x, w = s >> 5, l = s & 31;
      const bool valid = s < nmax;
      const int u = t.slots[s].unit;
      const bool start = valid && (s == 0 || u != t.slots[s - 1].unit);
      const unsigned bal = __ballot_sync(0xffffffffu, start);
      if (l == 0) t.sh[w] = __popc(bal);
      asm volatile("bar.sync 2, %0;" ::"n"(MT) : "memory");
      int before = 0;
      for (int k = 0; k < w; k++) before += (int)t.sh[k];
      const int seg = before + __popc(bal & (0xffffffffu >> (31 - l))) - 1;
      const int pr = s + h * seg;
      const bool fits = valid && pr < MT;
      // the tile's last pixel: the next one is missing or would not fit
      const bool valid1 = s + 1 < nmax;
      const int pr1 = s + 1 + h * (seg + ((valid1 && t.slots[s + 1].unit != u) ? 1 : 0));
      t.prow[s] = pr;
      if (fits) {
        const PixSlot ps = t.slots[s];
        t.wrow[pr + h] = make_int2(ps.unit, ps.i);
        if (start)
          for (int k = 1; k <= h; k++)
            t.wrow[pr + h - k] = make_int2(ps.i - k >= 0 ? ps.unit : -1, ps.i - k);
        if (!valid1 || pr1 >= MT) {
          t.flag[1] = s + 1;
          t.flag[2] = pr + 1;
          t.flag[3] = pr + 1 + h;
        }
      }
    }
  };
  // The schedule of step t + 1 (front sizes, this CTA's share, its first
  // tile's slots) needs no decoded data, so it is computed between arriving
  // at the grid barrier after step t and waiting for the others: the last
  // warp arrives (its release waits for the CTA's writes of step t to
  // reach GPU scope) while the other warps compute the schedule.
  const int NS = (int)blockDim.x - 32;
  if (pr) ck = clock64();
  int F = front_scan(a.units, a.n_units, 0, h, a.sched, t.pre, t.sh, (int)blockDim.x);
  tick(0);
  long long lo = (long long)F * blockIdx.x / G, hi = (long long)F * (blockIdx.x + 1) / G;
  if (lo < hi) {
    if constexpr (SHEAR) fill_slots_shear(0, lo, (int)min((long long)MT, hi - lo), (int)blockDim.x);
    else fill_slots(0, lo, (int)min((long long)MT, hi - lo), (int)blockDim.x);
  }
  __syncthreads();
  tick(1);
  for (int step = 0; step < a.T; step++) {
    for (long long base = lo; base < hi;) {
      int n = (int)min((long long)MT, hi - base);
      if (base != lo) {  // further tiles of a large share
        if constexpr (SHEAR) fill_slots_shear(step, base, n, (int)blockDim.x);
        else fill_slots(step, base, n, (int)blockDim.x);
        __syncthreads();
      }
      if constexpr (SHEAR) n = t.flag[1];
      // A CTA with at most one pixel per warp codes with whole warps (lower
      // latency per pixel); otherwise two pixels per warp.  Both give the
      // same tables (see cdf_fix).  Lane l of warp w copies the stream record
      // of the warp's l-th pixel into shared memory ahead of the network,
      // asynchronously (no register waits for it, so its round trip overlaps
      // the gather's); after the network, the 12 stream bytes from the
      // record's pos + 8, read only when the pixel is done.
      const bool wide = n <= NW;
      const int sl = wide ? group_slot<32, NW>(warp, lane) : group_slot<kGW, NW>(warp, lane);
      if (!SAMPLE && sl < n) {
        const StreamRec* r = a.st + t.slots[sl].aux;
        cp_async16(t.rec + sl, r);
        cp_async16(&t.rec[sl].pos, &r->pos);
      }
      if (pr) pc[5] += 1;
      tick(1);
      bool net_ok;
      if constexpr (SHEAR) {
        const long long c0 = pc != nullptr && threadIdx.x == 0 ? clock64() : 0;
        tc_gather_shear_win(a.units, t.wrow, a.ring, d, t.tc, step, t.flag[3]);
        __syncthreads();
        if (pc != nullptr && threadIdx.x == 0) pc[13] += clock64() - c0;
        net_ok = tc_network<NT>(d, t.tc, t.flag[2], pc, true);
      } else {
        net_ok = tile_network<PREC, true, NT>(a.m, a.units, t, n, pc);
      }
      // an MMA wait that timed out: record it and release every CTA from
      // the grid barrier (this one leaves its loop at its next wait)
      if (!net_ok && threadIdx.x == 0) {
        set_status(a.status, ST_TIMEOUT);
        atomicOr(a.bar, kBarPoison);
      }
      if constexpr (SAMPLE) {
        if (wide) sample_tile<32, NW, SHEAR>(a, t, n);
        else sample_tile<kGW, NW, SHEAR>(a, t, n);
        __syncthreads();
        tick(3);
        base += n;
        continue;
      }
      cp_async_wait_all();
      if (sl < n) {
        const unsigned long long w0 = (t.rec[sl].pos + 8ull) & ~3ull, end = t.rec[sl].end;
#pragma unroll
        for (int q = 0; q < 3; q++) {
          const unsigned long long wa = w0 + 4ull * q;
          cp_async4(t.win + 4 * sl + q, a.in + (wa < end ? wa : 0ull), wa < end);
        }
      }
      __syncwarp();  // the warp's records are visible to all its lanes
      tick(2);
      if (wide) code_tile<32, NW, SHEAR, PROF>(a, t, n, pc);
      else code_tile<kGW, NW, SHEAR, PROF>(a, t, n, pc);
      __syncthreads();
      tick(3);
      base += n;
    }
    if (step + 1 == a.T) break;
    const unsigned target = (unsigned)step + 1u;
    if ((int)threadIdx.x >= NS) {
      if (G > 1 && (int)threadIdx.x == NS) grid_arrive(a.bar);
    } else {
      F = front_scan(a.units, a.n_units, step + 1, h, a.sched, t.pre, t.sh, NS);
      tick(0);
      lo = (long long)F * blockIdx.x / G;
      hi = (long long)F * (blockIdx.x + 1) / G;
      if (lo < hi) {
        if constexpr (SHEAR) fill_slots_shear(step + 1, lo, (int)min((long long)MT, hi - lo), NS);
        else fill_slots(step + 1, lo, (int)min((long long)MT, hi - lo), NS);
      }
      tick(1);
    }
    if (G > 1) {
      if (!grid_wait(a.bar, G, target, a.status, t.flag, a.spin_limit)) break;
    } else {
      __syncthreads();
    }
    if ((int)threadIdx.x >= NS) {
      F = t.pre[a.n_units];
      lo = (long long)F * blockIdx.x / G;
      hi = (long long)F * (blockIdx.x + 1) / G;
    }
    tick(4);
    if (stamp && blockIdx.x == 0 && step + 1 < a.n_times) a.times[step + 1] = global_ns();
  }
  if (stamp && a.T < a.n_times) atomicMax(a.times + a.T, global_ns());
  if (pr) {
    for (int i = 0; i < 16; i++)
      if (i != 6 && i != 7) atomicAdd(a.prof + i, (unsigned long long)pc[i]);
    atomicAdd(a.prof + 6, 1ull);
    if (blockIdx.x == 0) atomicAdd(a.prof + 7, (unsigned long long)a.T);
  }
  if constexpr (PREC == PREC_BF16) tc_teardown(t.tc);
}

}  // namespace nlc
