// Device helpers shared by the codec kernels: unit lookup, block scans, the
// warp-level rANS decoder, the per-stream rANS encoder and the tile pipeline
// (gather -> local network) in shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nlc_common.cuh"
#include "nlc_kernels.cuh"
#include "nlc_model.cuh"
#include "nlc_tc.cuh"

namespace nlc {

constexpr int kMT = 64;  // pixels per tile of the FP32 pipeline

// ---------------------------------------------------------------------
// Shared helpers
// ---------------------------------------------------------------------
__device__ __forceinline__ int find_unit_px(const Unit* units, int n, long long q) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (units[mid].px_base <= q) lo = mid; else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int find_unit_stream(const Unit* units, int n, int s) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (units[mid].stream_base <= s) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Barrier of the first nt threads of the CTA (nt a multiple of 32): the whole
// CTA's __syncthreads when nt is its size, else named barrier 1.
__device__ __forceinline__ void part_sync(int nt) {
  if (nt == (int)blockDim.x) __syncthreads();
  else asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");
}

// Exclusive scan of one int per thread over the first nt threads of the CTA
// (nt a multiple of 32, only they call it); returns the exclusive prefix,
// writes the total to *total.
__device__ __forceinline__ long long block_excl_scan(long long v, long long* sh, long long* total,
                                                     int nt) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = nt >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) sh[warp] = x;
  part_sync(nt);
  if (warp == 0) {
    long long y = lane < nw ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long t = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += t;
    }
    if (lane < nw) sh[lane] = y;
  }
  part_sync(nt);
  long long excl = x - v + (warp > 0 ? sh[warp - 1] : 0);
  *total = sh[nw - 1];
  part_sync(nt);
  return excl;
}
__device__ __forceinline__ long long block_excl_scan(long long v, long long* sh, long long* total) {
  return block_excl_scan(v, sh, total, (int)blockDim.x);
}

// Fronts of all units at global step t: pre[u] = exclusive prefix of the
// front sizes, pre[n_units] = total.  Requires n_units + 1 ints of smem.
// Computed by (and returned to) the first nt threads of the CTA.
__device__ __forceinline__ int front_scan(const Unit* __restrict__ units, int n_units, int t,
                                          int h, int sched, int* pre, long long* sh, int nt) {
  const int per = (n_units + nt - 1) / nt;
  const int u0 = threadIdx.x * per, u1 = min(u0 + per, n_units);
  long long sum = 0;
  for (int u = u0; u < u1; u++) {
    int c = unit_front(units[u], t, h, sched).n;
    pre[u] = c;
    sum += c;
  }
  long long total;
  long long run = block_excl_scan(sum, sh, &total, nt);
  for (int u = u0; u < u1; u++) {
    int c = pre[u];
    pre[u] = (int)run;
    run += c;
  }
  if (threadIdx.x == 0) pre[n_units] = (int)total;
  part_sync(nt);
  return (int)total;
}

// ---------------------------------------------------------------------
// rANS: warp-level decoder of one stream position and the per-stream
// encoder (byte-wise renormalisation, state in [2^23, 2^31)).
// ---------------------------------------------------------------------
// Coding groups of the codec kernels: 16 lanes (half a warp) per pixel.
constexpr int kGW = 16;
constexpr int kGroups = kThreads / kGW;

// Decoder of one rANS stream position, held uniformly by a coding group.
// The next 8 stream bytes (a pixel consumes at most 6) are held in two
// registers; w2, w3 hold the 8 after them, from which the state written back
// for the stream's next pixel takes its 8 bytes.
struct GroupRansDec {
  uint32_t x;
  uint32_t lo, hi;  // bytes pos .. pos+7, little-endian packed
  uint32_t w2, w3;  // bytes pos+8 .. pos+15
  int used;
  int avail;        // bytes of the stream left from pos, at most 8
  bool bad;

  // w2, w3 from the three aligned words at (pos + 8) & ~3 (a word is read
  // only if it starts before the stream's end, so none outside its container).
  __device__ __forceinline__ void set_window(const uint32_t* v, unsigned long long pos) {
    const uint32_t sh = 8u * (uint32_t)((pos + 8ull) & 3ull);
    w2 = __funnelshift_r(v[0], v[1], sh);
    w3 = __funnelshift_r(v[1], v[2], sh);
  }
  // The 8 bytes at pos + used (used <= 6 for a valid pixel).
  __device__ __forceinline__ void next_bytes(uint32_t& n0, uint32_t& n1) const {
    if (used < 4) {
      const uint32_t s = 8u * (uint32_t)used;
      n0 = __funnelshift_r(lo, hi, s);
      n1 = __funnelshift_r(hi, w2, s);
    } else {
      const uint32_t s = 8u * (uint32_t)(used - 4);
      n0 = __funnelshift_r(hi, w2, s);
      n1 = __funnelshift_r(w2, w3, s);
    }
  }
  __device__ __forceinline__ void set_avail(unsigned long long pos, unsigned long long end) {
    avail = pos < end ? (int)min(end - pos, 8ull) : 0;
  }

  __device__ __forceinline__ void load_bytes(const uint8_t* base, unsigned long long pos,
                                             unsigned long long end) {
    lo = hi = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const unsigned long long p = pos + (unsigned long long)k;
      const uint32_t v = p < end ? (uint32_t)base[p] : 0u;
      if (k < 4) lo |= v << (8 * k);
      else hi |= v << (8 * (k - 4));
    }
    set_avail(pos, end);
    used = 0;
  }
  // With slot = x mod 2^16 and the decoded symbol's cum_s <= slot < cum_{s+1}:
  // x = freq (x >> 16) + slot - cum_s, then shift bytes in while x < 2^23.
  __device__ __forceinline__ void advance(uint32_t slot, uint32_t c0, uint32_t c1) {
    x = (c1 - c0) * (x >> 16) + slot - c0;
    for (int it = 0; it < 3 && x < kRansL; it++) {
      const uint32_t bt = used < 4 ? (lo >> (8 * used)) & 0xFFu
                                   : used < 8 ? (hi >> (8 * (used - 4))) & 0xFFu : 0u;
      if (used >= avail) bad = true;
      x = (x << 8) | bt;
      used++;
    }
    if (x < kRansL) bad = true;
  }
  // One symbol from an explicit table.
  template <int GW>
  __device__ __forceinline__ int decode_table(const TableScratch& ws, int lane) {
    const uint32_t slot = x & 0xFFFFu;
    const int s = table_search<GW>(ws, slot, lane);
    advance(slot, cum_at<GW>(ws, s), cum_at<GW>(ws, s + 1));
    return s;
  }
};

// Encodes symbols k = nsym-1 .. 0 (packed start | freq << 16) ending at
// slot_end; returns the stream length.  Layout: 4-byte big-endian final
// state, then the emitted bytes in reverse emission order.
template <class Get>
__device__ __forceinline__ int rans_encode_stream(Get get, long long nsym, uint8_t* slot_end) {
  uint8_t* w = slot_end;
  uint32_t x = kRansL;
  for (long long k = nsym - 1; k >= 0; k--) {
    const uint32_t e = get(k);
    const uint32_t start = e & 0xFFFFu, f = e >> 16;
    const uint32_t xmax = ((kRansL >> 16) << 8) * f;
    while (x >= xmax) {
      *--w = (uint8_t)(x & 0xFFu);
      x >>= 8;
    }
    x = ((x / f) << 16) + (x % f) + start;
  }
  *--w = (uint8_t)x;
  *--w = (uint8_t)(x >> 8);
  *--w = (uint8_t)(x >> 16);
  *--w = (uint8_t)(x >> 24);
  return (int)(slot_end - w);
}

// ---------------------------------------------------------------------
// Tile pipeline (FP32 SIMT network) shared by encode, decode and forward.
// ---------------------------------------------------------------------
struct TileSmem {
  float* Wt;
  float* A;
  float* B1;
  float* U0;
  WarpScratch* ws;
  PixSlot* slots;
  int* pre;
  StreamRec* rec;  // decoder: the tile's stream records (kTileMax)
  uint32_t* win;   // decoder: per pixel, the 12 stream bytes from pos + 8, word-aligned
  int* prow;       // sheared wavefront decoder: output row of the tile's pixel s
  int* rofs;       // sheared wavefront decoder: ring byte offset of the tile's pixel s
  int2* wrow;      // sheared wavefront decoder: (unit, unit row) of window row rho
  long long* sh;
  long long* pc;  // 16 profiling accumulators (thread 0 only)
  int* flag;
  TcSmem tc;
};

// Network outputs of the tile's m-th pixel.
__device__ __forceinline__ const float* tile_params(const TileSmem& t, const Dims& d, int m) {
  return t.U0 + (size_t)m * d.ldP;
}

// Shared memory of the tile pipeline with `groups` coding groups (and, for
// the decoder, the tile's stream records and windows).
__host__ __device__ inline size_t tile_smem_bytes(const Dims& d, int n_pre, int groups = kGroups,
                                                  bool dec = false) {
  size_t bytes;
  if (d.prec == PREC_BF16) {
    bytes = tc_smem_bytes(d);
  } else {
    SimtPlan pl = simt_plan(d, (int)simt_floats(d), kMT);
    bytes = (size_t)pl.end * 4;
  }
  bytes = (bytes + 15) & ~(size_t)15;
  bytes += sizeof(WarpScratch) * groups;
  if (dec) bytes += (sizeof(StreamRec) + 4 * sizeof(uint32_t) + 2 * sizeof(int)) * kTileMax +
                    sizeof(int2) * kWinRows;
  bytes += sizeof(PixSlot) * kTileMax;
  bytes += sizeof(long long) * (33 + 16);
  bytes += sizeof(int) * (n_pre + 1 + 4);
  return (bytes + 15) & ~(size_t)15;
}

__device__ __forceinline__ TileSmem carve(const Dims& d, unsigned char* smem, int n_pre,
                                          int groups = kGroups, bool dec = false) {
  TileSmem t;
  size_t off;
  if (d.prec == PREC_BF16) {
    t.tc = tc_carve(d, smem);
    off = tc_smem_bytes(d);
    t.Wt = t.A = t.B1 = nullptr;
    t.U0 = t.tc.P;
  } else {
    SimtPlan pl = simt_plan(d, (int)simt_floats(d), kMT);
    float* f = reinterpret_cast<float*>(smem);
    t.Wt = f + pl.w_off;
    t.A = f + pl.a_off;
    t.B1 = f + pl.b1_off;
    t.U0 = f + pl.u0_off;
    off = (size_t)pl.end * 4;
  }
  off = (off + 15) & ~(size_t)15;
  t.ws = reinterpret_cast<WarpScratch*>(smem + off);
  off += sizeof(WarpScratch) * groups;
  t.rec = nullptr;
  t.win = nullptr;
  t.prow = nullptr;
  t.rofs = nullptr;
  t.wrow = nullptr;
  if (dec) {
    t.rec = reinterpret_cast<StreamRec*>(smem + off);
    off += sizeof(StreamRec) * kTileMax;
    t.win = reinterpret_cast<uint32_t*>(smem + off);
    off += 4 * sizeof(uint32_t) * kTileMax;
    t.wrow = reinterpret_cast<int2*>(smem + off);
    off += sizeof(int2) * kWinRows;
    t.prow = reinterpret_cast<int*>(smem + off);
    off += sizeof(int) * kTileMax;
    t.rofs = reinterpret_cast<int*>(smem + off);
    off += sizeof(int) * kTileMax;
  }
  t.slots = reinterpret_cast<PixSlot*>(smem + off);
  off += sizeof(PixSlot) * kTileMax;
  t.sh = reinterpret_cast<long long*>(smem + off);
  off += sizeof(long long) * 33;
  t.pc = reinterpret_cast<long long*>(smem + off);
  off += sizeof(long long) * 16;
  t.pre = reinterpret_cast<int*>(smem + off);
  t.flag = t.pre + n_pre + 1;
  (void)n_pre;
  return t;
}

template <int PREC>
__device__ __forceinline__ constexpr int tile_size() { return PREC == PREC_BF16 ? kTcM : kMT; }

template <int PREC>
__device__ __forceinline__ void load_weights(const DeviceModel& m, TileSmem& t) {
  if constexpr (PREC == PREC_BF16) {
    tc_load_weights(m.d, m.w, t.tc);
  } else {
    const int n = m.w.simt_floats;
    for (int i = threadIdx.x; i < n; i += blockDim.x) t.Wt[i] = m.w.simt[i];
  }
}

// gather + network for the slots of the tile; P[m][NOp] lands in t.U0.
// With pc non-null (BF16), thread 0 adds its gather cycles to pc[13] and the
// network's sub-phases to pc[14], pc[15] (shared-memory accumulators).
// Returns false (in every thread) if an MMA completion wait timed out.
template <int PREC, bool kCoherent, int NT = kThreads>
__device__ __forceinline__ bool tile_network(const DeviceModel& m, const Unit* units, TileSmem& t,
                                             int n_valid, long long* pc = nullptr) {
  if constexpr (PREC == PREC_BF16) {
    const long long c0 = pc != nullptr && threadIdx.x == 0 ? clock64() : 0;
    if (m.d.shear) tc_gather_shear_px<kCoherent>(units, t.slots, m.d, t.tc, n_valid);
    else tc_gather<kCoherent>(units, t.slots, m.d, t.tc, n_valid);
    __syncthreads();
    if (pc != nullptr && threadIdx.x == 0) pc[13] += clock64() - c0;
    return tc_network<NT>(m.d, t.tc, n_valid, pc);
  } else {
    gather_f32<kMT, kCoherent>(units, t.slots, m.d.h, t.U0);
    __syncthreads();
    network_simt_run<kMT>(m.d, t.Wt, t.A, t.B1, t.U0);
    return true;
  }
}


__device__ __forceinline__ int unit_streams(const Unit& U, int layout) {
  return layout == 1 ? U.Hu : 1;
}

inline int grid_for(long long work, int per, int cap) {
  long long g = (work + per - 1) / per;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace nlc
