// Codec kernels of the nlc library (sm_103a) other than the tile pipeline:
// weight packing, the per-stream rANS encoder, container pack/parse and the
// stage-level entry points used by the parity tests.
#include "nlc_tile.cuh"

namespace nlc {

// ---------------------------------------------------------------------
// Weight packing
// ---------------------------------------------------------------------
// Canonical FP32 layout: W0[C][F] b0[C] {W1[C][C] b1 W2[C][C] b2}xR WH[NO][C] bH[NO].
__global__ void repack_simt_kernel(Dims d, const float* __restrict__ w, float* __restrict__ out) {
  const int C = d.C, F = d.F, NO = d.NO, NOp = d.NOp;
  const long long total = (long long)simt_floats(d);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long r = e;
    long long src_base = 0;
    float v = 0.f;
    if (r < (long long)F * C) {  // W0T[f][c] = W0[c][f]
      int f = (int)(r / C), c = (int)(r % C);
      v = w[(long long)c * F + f];
    } else {
      r -= (long long)F * C;
      src_base = (long long)F * C;
      if (r < C) {
        v = w[src_base + r];
      } else {
        r -= C;
        src_base += C;
        bool done = false;
        for (int b = 0; b < d.R && !done; b++) {
          for (int part = 0; part < 2 && !done; part++) {
            if (r < (long long)C * C) {  // WT[k][n] = W[n][k]
              int k = (int)(r / C), n = (int)(r % C);
              v = w[src_base + (long long)n * C + k];
              done = true;
            } else {
              r -= (long long)C * C;
              src_base += (long long)C * C;
              if (r < C) { v = w[src_base + r]; done = true; }
              else { r -= C; src_base += C; }
            }
          }
        }
        if (!done) {
          if (r < (long long)C * NOp) {  // WHT[k][n] = WH[n][k], zero pad n >= NO
            int k = (int)(r / NOp), n = (int)(r % NOp);
            v = n < NO ? w[src_base + (long long)n * C + k] : 0.f;
          } else {
            r -= (long long)C * NOp;
            src_base += (long long)NO * C;
            v = r < NO ? w[src_base + r] : 0.f;
          }
        }
      }
    }
    out[e] = v;
  }
}

// Order-independent 64-bit content hash of (dims, weights): XOR of a
// splitmix64 finaliser over (index, word).
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void hash_kernel(Dims d, const float* __restrict__ w, int n, unsigned long long* out) {
  __shared__ unsigned long long part[kThreads];
  unsigned long long hsh = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    hsh ^= mix64(((unsigned long long)i << 32) ^ __float_as_uint(w[i]));
  part[threadIdx.x] = hsh;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = mix64(((unsigned long long)d.h << 48) ^ ((unsigned long long)d.C << 32) ^
                                 ((unsigned long long)d.R << 16) ^ (unsigned long long)d.K);
    t ^= mix64(0xABCDull ^ (unsigned long long)prec_code(d));
    for (int i = 0; i < (int)blockDim.x; i++) t ^= part[i];
    *out = t;
  }
}

// BF16 operand tiles for the tensor-core path, in the canonical no-swizzle
// K-major layout (see nlc_tc.cuh): W0 (C x Fp, scaled by 1/255, zero for
// k >= F), W1_r, W2_r (C x C), WH (NOp x C, zero rows n >= NO); biases FP32.
__global__ void repack_umma_kernel(Dims d, const float* __restrict__ w, uint16_t* __restrict__ umma,
                                   float* __restrict__ bias) {
  const int C = d.C, F = d.F, Fp = d.Fp, NO = d.NO, NOp = d.NOp;
  const long long total = (long long)umma_halves(d);
  const long long gstride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += gstride) {
    long long o = e;
    int Kd;
    long long wbase;  // canonical offset of the FP32 matrix
    int kind;         // 0 W0, 1 hidden, 2 head, 3 sheared W0
    int dd = 0;       // sheared: window row (0 = top, h = the pixel's own row)
    const long long plain = (long long)umma_plain_halves(d);
    int c_lo = 0;  // sheared: first 8-feature chunk of window row dd's MMAs
    if (o >= plain) {
      o -= plain;
      int ks = 0;
      dd = 0;
      while (dd < d.h && o >= (long long)shear_tile_off(d, dd + 1)) dd++;
      o -= shear_tile_off(d, dd);
      shear_krange(d.h, d.Ws, dd, c_lo, ks);
      Kd = 16 * ks; wbase = 0; kind = 3;
    } else if (o < (long long)C * Fp) {
      Kd = Fp; wbase = 0; kind = 0;
    } else {
      o -= (long long)C * Fp;
      const long long blk = 2LL * C * C;
      if (o < blk * d.R) {
        const int r = (int)(o / blk);
        long long rem = o % blk;
        const int part = (int)(rem / ((long long)C * C));
        o = rem % ((long long)C * C);
        Kd = C; kind = 1;
        wbase = (long long)C * F + C + (long long)r * (2LL * C * C + 2 * C) +
                (long long)part * (C * C + C);
      } else {
        o -= blk * d.R;
        Kd = C; kind = 2;
        wbase = (long long)C * F + C + (long long)d.R * (2LL * C * C + 2 * C);
      }
    }
    const int core = (int)(o / 64), within = (int)(o % 64);
    const int rb = core / (Kd / 8), kb = core % (Kd / 8);
    const int r = rb * 8 + within / 8;
    int k = kb * 8 + within % 8;
    float v;
    if (kind == 0) v = k < F ? __fdiv_rn(w[(long long)r * F + k], 255.f) : 0.f;
    else if (kind == 3) {
      k += 8 * c_lo;  // feature of the window row
      // window row dd, window column q = k / 3 (channel k % 3): the pixel at
      // row offset dy = dd - h and column offset dx = q - Ws + (h+1)(h - dd)
      // (the sheared column t - Ws + q of row i + dy, t = j + (h+1) i); its
      // weight is the tap's (Fig. 5), 0 where the window holds no tap
      const int h = d.h, q = k / 3, c = k % 3;
      const int dy = dd - h, dx = q - d.Ws + (h + 1) * (h - dd);
      int p = -1;
      if (k < 3 * d.Ws) {
        if (dy < 0 && dx >= -h && dx <= h) p = (dy + h) * (2 * h + 1) + (dx + h);
        if (dy == 0 && dx >= -h && dx <= -1) p = h * (2 * h + 1) + (dx + h);
      }
      v = p >= 0 ? __fdiv_rn(w[(long long)r * F + 3 * p + c], 255.f) : 0.f;
    } else if (kind == 1) v = w[wbase + (long long)r * C + k];
    else v = r < NO ? w[wbase + (long long)r * C + k] : 0.f;
    umma[e] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
  }
  // biases: b0 {b1 b2}xR bH(padded)
  const int nb = (int)bias_floats(d);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nb; e += gstride) {
    int i = (int)e;
    float v;
    if (i < C) {
      v = w[(long long)C * F + i];
    } else if (i < C + 2 * d.R * C) {
      const int j = i - C, r = j / (2 * C), part = (j % (2 * C)) / C, c = j % C;
      const long long base = (long long)C * F + C + (long long)r * (2LL * C * C + 2 * C) +
                             (long long)part * (C * C + C) + (long long)C * C;
      v = w[base + c];
    } else {
      const int n = i - C - 2 * d.R * C;
      const long long base = (long long)C * F + C + (long long)d.R * (2LL * C * C + 2 * C) +
                             (long long)NO * C;
      v = n < NO ? w[base + n] : 0.f;
    }
    bias[i] = v;
  }
}

cudaError_t launch_repack_umma(const Dims& d, const float* w, uint16_t* umma, float* bias,
                               cudaStream_t s) {
  repack_umma_kernel<<<64, 256, 0, s>>>(d, w, umma, bias);
  return cudaGetLastError();
}

cudaError_t launch_repack(const Dims& d, const float* w, float* simt, uint16_t* umma, float* bias,
                          unsigned long long* hash, int n_w, cudaStream_t s) {
  repack_simt_kernel<<<64, 256, 0, s>>>(d, w, simt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (d.prec == PREC_BF16) {
    e = launch_repack_umma(d, w, umma, bias, s);
    if (e != cudaSuccess) return e;
  }
  if (hash == nullptr) return cudaSuccess;
  return launch_hash(d, w, n_w, hash, s);
}

cudaError_t launch_hash(const Dims& d, const float* w, int n_w, unsigned long long* hash,
                        cudaStream_t s) {
  hash_kernel<<<1, kThreads, 0, s>>>(d, w, n_w, hash);
  return cudaGetLastError();
}

__global__ void rans_enc_kernel(const Unit* __restrict__ units, int n_units, int n_streams,
                                int layout, const uint32_t* __restrict__ stage,
                                uint8_t* __restrict__ scratch, int32_t* __restrict__ lens) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_streams) return;
  const Unit U = units[find_unit_stream(units, n_units, s)];
  long long p0, np;
  if (layout == 1) {
    p0 = U.px_base + (long long)(s - U.stream_base) * U.Wu;
    np = U.Wu;
  } else {
    p0 = U.px_base;
    np = (long long)U.Hu * U.Wu;
  }
  const long long sym0 = 3 * p0, nsym = 3 * np;
  uint8_t* slot_end = scratch + 2 * sym0 + 4LL * s + 2 * nsym + 4;
  const uint32_t* st = stage + sym0;
  lens[s] = rans_encode_stream([&](long long k) { return st[k]; }, nsym, slot_end);
}

// Sum of the stream lengths of each unit (one warp per unit).
__global__ void unit_sum_kernel(const Unit* __restrict__ units, int n_units, int layout,
                                const int32_t* __restrict__ lens,
                                unsigned long long* __restrict__ unit_bytes) {
  const int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (u >= n_units) return;
  const Unit U = units[u];
  const int ns = unit_streams(U, layout);
  unsigned long long s = 0;
  for (int k = lane; k < ns; k += 32) s += (unsigned)lens[U.stream_base + k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) unit_bytes[u] = s;
}

// Container plan (one thread): offsets of the containers and of the units'
// stream data; flags a capacity overflow.
__global__ void pack_plan_kernel(const ImageRec* __restrict__ images, int n_images, int layout,
                                 int patch, const unsigned long long* __restrict__ unit_bytes,
                                 unsigned long long* __restrict__ unit_off,
                                 unsigned long long* __restrict__ offsets, unsigned long long cap,
                                 int* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  unsigned long long off = 0;
  for (int i = 0; i < n_images; i++) {
    const ImageRec I = images[i];
    const int lw = len_width(I.H, I.W, patch, layout);
    unsigned long long o = off + kHeaderBytes + (unsigned long long)lw * I.n_streams;
    for (int u = I.unit_base; u < I.unit_base + I.n_units; u++) {
      unit_off[u] = o;
      o += unit_bytes[u];
    }
    offsets[i] = off;
    off += ((o - off) + 15ull) & ~15ull;
  }
  offsets[n_images] = off;
  if (off > cap) set_status(status, ST_CAPACITY);
}

// Copy of the streams into the containers, length tables and headers (one
// block per unit).
__global__ void pack_copy_kernel(DeviceModel m, const Unit* __restrict__ units, int n_units,
                                 const ImageRec* __restrict__ images, int n_images, int layout,
                                 int patch, const int32_t* __restrict__ lens,
                                 const uint8_t* __restrict__ scratch,
                                 const unsigned long long* __restrict__ unit_off,
                                 unsigned long long* __restrict__ soff,
                                 const unsigned long long* __restrict__ offsets,
                                 unsigned long long cap, uint8_t* __restrict__ out) {
  __shared__ long long sh[33];
  const int u = blockIdx.x;
  if (u >= n_units || offsets[n_images] > cap) return;
  const Unit U = units[u];
  const ImageRec I = images[U.image];
  const unsigned long long cbase = offsets[U.image];
  const int ns = unit_streams(U, layout);
  long long run = 0;
  for (int c0 = 0; c0 < ns; c0 += blockDim.x) {
    const int k = c0 + threadIdx.x;
    const long long len = k < ns ? lens[U.stream_base + k] : 0;
    long long total;
    long long ex = block_excl_scan(len, sh, &total);
    if (k < ns) {
      soff[U.stream_base + k] = unit_off[u] + (unsigned long long)(run + ex);
      const int sidx = U.stream_base + k - I.stream_base;
      uint8_t* lp = out + cbase + kHeaderBytes;
      if (len_width(I.H, I.W, patch, layout) == 2)
        reinterpret_cast<uint16_t*>(lp)[sidx] = (uint16_t)len;
      else
        reinterpret_cast<uint32_t*>(lp)[sidx] = (uint32_t)len;
    }
    run += total;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = warp; k < ns; k += nw) {
    const int s = U.stream_base + k;
    long long p0, np;
    if (layout == 1) { p0 = U.px_base + (long long)k * U.Wu; np = U.Wu; }
    else { p0 = U.px_base; np = (long long)U.Hu * U.Wu; }
    const uint8_t* slot_end = scratch + 6 * p0 + 4LL * s + 6 * np + 4;
    const int len = lens[s];
    const uint8_t* src = slot_end - len;
    uint8_t* dst = out + soff[s];
    for (int b = lane; b < len; b += 32) dst[b] = src[b];
  }
  if (threadIdx.x == 0 && u == I.unit_base) {
    uint8_t* h = out + cbase;
    *reinterpret_cast<uint32_t*>(h + 0) = kMagic;
    h[4] = (uint8_t)kVersion;
    h[5] = (uint8_t)m.d.h;
    h[6] = (uint8_t)layout;
    h[7] = (uint8_t)prec_code(m.d);
    *reinterpret_cast<uint32_t*>(h + 8) = (uint32_t)I.H;
    *reinterpret_cast<uint32_t*>(h + 12) = (uint32_t)I.W;
    *reinterpret_cast<uint32_t*>(h + 16) = (uint32_t)patch;
    *reinterpret_cast<uint32_t*>(h + 20) = (uint32_t)I.n_streams;
    *reinterpret_cast<unsigned long long*>(h + 24) = *m.hash;
  }
  // zero padding after the image's last unit
  if (u == I.unit_base + I.n_units - 1) {
    unsigned long long end = unit_off[u];
    for (int k = 0; k < ns; k++) end += (unsigned)lens[U.stream_base + k];
    const unsigned long long cend = offsets[U.image + 1];
    for (unsigned long long p = end + threadIdx.x; p < cend; p += blockDim.x) out[p] = 0;
  }
}

// Header and padding of images without units (H or W = 0).
__global__ void pack_empty_kernel(DeviceModel m, const ImageRec* __restrict__ images, int n_images,
                                  int layout, int patch, const unsigned long long* offsets,
                                  unsigned long long cap, uint8_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_images || offsets[n_images] > cap) return;
  const ImageRec I = images[i];
  if (I.n_units > 0) return;
  uint8_t* h = out + offsets[i];
  for (int b = 0; b < kHeaderBytes; b++) h[b] = 0;
  *reinterpret_cast<uint32_t*>(h + 0) = kMagic;
  h[4] = (uint8_t)kVersion;
  h[5] = (uint8_t)m.d.h;
  h[6] = (uint8_t)layout;
  h[7] = (uint8_t)prec_code(m.d);
  *reinterpret_cast<uint32_t*>(h + 8) = (uint32_t)I.H;
  *reinterpret_cast<uint32_t*>(h + 12) = (uint32_t)I.W;
  *reinterpret_cast<uint32_t*>(h + 16) = (uint32_t)patch;
  *reinterpret_cast<uint32_t*>(h + 20) = 0u;
  *reinterpret_cast<unsigned long long*>(h + 24) = *m.hash;
}

cudaError_t launch_encode(const DeviceModel& m, const CodecBufs& b, int layout, int patch,
                          uint8_t* out, unsigned long long cap, unsigned long long* d_offsets,
                          int sm_count, cudaStream_t s) {
  cudaError_t e;
  if (b.n_units > 0) {
    if ((e = launch_enc_tables(m, b, sm_count, s)) != cudaSuccess) return e;
    rans_enc_kernel<<<grid_for(b.n_streams, 128, 1 << 20), 128, 0, s>>>(
        b.units, b.n_units, b.n_streams, layout, b.stage, b.scratch, b.lens);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    unit_sum_kernel<<<grid_for((long long)b.n_units * 32, 256, 1 << 20), 256, 0, s>>>(
        b.units, b.n_units, layout, b.lens, b.unit_bytes);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  pack_plan_kernel<<<1, 32, 0, s>>>(b.images, b.n_images, layout, patch, b.unit_bytes, b.unit_off,
                                    d_offsets, cap, b.status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (b.n_units > 0) {
    pack_copy_kernel<<<b.n_units, 256, 0, s>>>(m, b.units, b.n_units, b.images, b.n_images, layout,
                                               patch, b.lens, b.scratch, b.unit_off, b.st_pos,
                                               d_offsets, cap, out);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  pack_empty_kernel<<<grid_for(b.n_images, 128, 1 << 20), 128, 0, s>>>(m, b.images, b.n_images,
                                                                       layout, patch, d_offsets,
                                                                       cap, out);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------
// Decoder: container parse
// ---------------------------------------------------------------------
__global__ void parse_header_kernel(DeviceModel m, const ImageRec* __restrict__ images,
                                    int n_images, int layout, int patch,
                                    const uint8_t* __restrict__ in,
                                    const unsigned long long* __restrict__ offsets,
                                    int* __restrict__ bad, int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_images) return;
  const ImageRec I = images[i];
  const unsigned long long o = offsets[i], o1 = offsets[i + 1];
  int err = 0;
  const int lw = len_width(I.H, I.W, patch, layout);
  if (o1 < o || o1 - o < kHeaderBytes + (unsigned long long)lw * I.n_streams || (o & 15ull)) {
    err = ST_CORRUPT;
  } else {
    const uint8_t* h = in + o;
    if (*reinterpret_cast<const uint32_t*>(h) != kMagic || h[4] != kVersion || h[5] != m.d.h ||
        h[6] != layout || *reinterpret_cast<const uint32_t*>(h + 8) != (uint32_t)I.H ||
        *reinterpret_cast<const uint32_t*>(h + 12) != (uint32_t)I.W ||
        *reinterpret_cast<const uint32_t*>(h + 16) != (uint32_t)patch ||
        *reinterpret_cast<const uint32_t*>(h + 20) != (uint32_t)I.n_streams)
      err = ST_CORRUPT;
    else if (h[7] != prec_code(m.d) || *reinterpret_cast<const unsigned long long*>(h + 24) != *m.hash)
      err = ST_WEIGHTS;
  }
  bad[i] = err;
  if (err) set_status(status, err);
}

__global__ void parse_lens_kernel(const Unit* __restrict__ units, int n_units,
                                  const ImageRec* __restrict__ images, int layout, int patch,
                                  const uint8_t* __restrict__ in,
                                  const unsigned long long* __restrict__ offsets,
                                  const int* __restrict__ bad, int32_t* __restrict__ lens,
                                  unsigned long long* __restrict__ unit_bytes) {
  const int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (u >= n_units) return;
  const Unit U = units[u];
  const ImageRec I = images[U.image];
  const int ns = unit_streams(U, layout);
  const bool ok = bad[U.image] == 0;
  const int lw = len_width(I.H, I.W, patch, layout);
  unsigned long long s = 0;
  for (int k = lane; k < ns; k += 32) {
    const int sidx = U.stream_base + k - I.stream_base;
    const uint8_t* lp = in + offsets[U.image] + kHeaderBytes;
    uint32_t len = 0u;
    if (ok)
      len = lw == 2 ? (uint32_t)reinterpret_cast<const uint16_t*>(lp)[sidx]
                    : reinterpret_cast<const uint32_t*>(lp)[sidx];
    lens[U.stream_base + k] = (int32_t)len;
    s += len;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) unit_bytes[u] = s;
}

__global__ void parse_plan_kernel(const ImageRec* __restrict__ images, int n_images, int layout,
                                  int patch, const unsigned long long* __restrict__ offsets,
                                  const unsigned long long* __restrict__ unit_bytes,
                                  unsigned long long* __restrict__ unit_off, int* __restrict__ bad,
                                  int* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < n_images; i++) {
    const ImageRec I = images[i];
    unsigned long long o = offsets[i] + kHeaderBytes +
                           (unsigned long long)len_width(I.H, I.W, patch, layout) * I.n_streams;
    for (int u = I.unit_base; u < I.unit_base + I.n_units; u++) {
      unit_off[u] = o;
      o += unit_bytes[u];
    }
    if (!bad[i] && o > offsets[i + 1]) {
      bad[i] = ST_CORRUPT;
      set_status(status, ST_CORRUPT);
    }
  }
}

__global__ void parse_streams_kernel(const Unit* __restrict__ units, int n_units, int layout,
                                     const uint8_t* __restrict__ in,
                                     const int32_t* __restrict__ lens,
                                     const unsigned long long* __restrict__ unit_off,
                                     const int* __restrict__ bad, StreamRec* __restrict__ st,
                                     int* status) {
  __shared__ long long sh[33];
  const int u = blockIdx.x;
  if (u >= n_units) return;
  const Unit U = units[u];
  const int ns = unit_streams(U, layout);
  const bool ok = bad[U.image] == 0;
  long long run = 0;
  for (int c0 = 0; c0 < ns; c0 += blockDim.x) {
    const int k = c0 + threadIdx.x;
    const long long len = k < ns ? lens[U.stream_base + k] : 0;
    long long total;
    long long ex = block_excl_scan(len, sh, &total);
    if (k < ns) {
      const int s = U.stream_base + k;
      const unsigned long long p = unit_off[u] + (unsigned long long)(run + ex);
      uint32_t x = 0;
      if (ok && len >= 4) {
        x = ((uint32_t)in[p] << 24) | ((uint32_t)in[p + 1] << 16) | ((uint32_t)in[p + 2] << 8) |
            (uint32_t)in[p + 3];
      }
      StreamRec r;
      r.pad = 0;
      if (!ok || len < 4 || x < kRansL || x >= (1u << 31)) {
        if (ok) set_status(status, ST_CORRUPT);
        r.x = kRansL;
        r.pos = r.end = p;
      } else {
        r.x = x;
        r.pos = p + 4;
        r.end = p + (unsigned long long)len;
      }
      // the stream's first 8 payload bytes (0 past its end)
      uint32_t w[2] = {0u, 0u};
      for (int q = 0; q < 8; q++) {
        const unsigned long long pq = r.pos + (unsigned long long)q;
        if (pq < r.end) w[q >> 2] |= (uint32_t)in[pq] << (8 * (q & 3));
      }
      r.b0 = w[0];
      r.b1 = w[1];
      st[s] = r;
    }
    run += total;
  }
}

cudaError_t launch_parse(const DeviceModel& m, const CodecBufs& b, const uint8_t* in,
                         const unsigned long long* d_offsets, int layout, int patch,
                         cudaStream_t s) {
  cudaError_t e;
  int* bad = reinterpret_cast<int*>(b.unit_bytes + b.n_units + 1);
  parse_header_kernel<<<grid_for(b.n_images, 128, 1 << 20), 128, 0, s>>>(
      m, b.images, b.n_images, layout, patch, in, d_offsets, bad, b.status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (b.n_units == 0) return cudaSuccess;
  parse_lens_kernel<<<grid_for((long long)b.n_units * 32, 256, 1 << 20), 256, 0, s>>>(
      b.units, b.n_units, b.images, layout, patch, in, d_offsets, bad, b.lens, b.unit_bytes);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  parse_plan_kernel<<<1, 32, 0, s>>>(b.images, b.n_images, layout, patch, d_offsets, b.unit_bytes,
                                     b.unit_off, bad, b.status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  parse_streams_kernel<<<b.n_units, 256, 0, s>>>(b.units, b.n_units, layout, in, b.lens,
                                                 b.unit_off, bad, b.st,
                                                 b.status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------
// Stage entry points for parity tests.
// ---------------------------------------------------------------------
__global__ void tables_kernel(int K, int NO, const float* __restrict__ params,
                              const uint8_t* __restrict__ pixels, long long n,
                              uint32_t* __restrict__ cum) {
  // the codec's 16-lane coding groups, two pixels per warp; lanes take the
  // boundaries gl, gl + 16, ... with all active components each
  __shared__ WarpScratch ws[kGroups];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int half = lane >> 4, gl = lane & (kGW - 1);
  for (long long q0 = ((long long)blockIdx.x * kWarps + warp) * 2; q0 < n;
       q0 += (long long)gridDim.x * kWarps * 2) {
    const long long q = q0 + half;
    const bool valid = q < n;
    const long long qe = valid ? q : q0;
    const int v[3] = {pixels[3 * qe], pixels[3 * qe + 1], pixels[3 * qe + 2]};
    WarpScratch& g = ws[2 * warp + half];
    CompState cs;
    comp_init<kGW>(params + qe * NO, K, gl, cs);
    for (int ch = 0; ch < 3; ch++) {
      int nact;
      const float mloc = channel_setup<kGW>(cs, K, ch, v[0], v[1], gl, g, nact);
      uint32_t* o = cum + (qe * 3 + ch) * 257;
      for (int b = gl; b < 257; b += kGW) {
        const uint32_t u = cum_fix(b >= 1 && b <= 255 ? cdf_fix(g, nact, edge_f(b), 0, 1) : 0, b);
        if (valid) o[b] = u;
      }
      if (ch < 2) comp_observe(cs, K, ch, mloc, v[ch], gl);
      __syncwarp();
    }
  }
}

cudaError_t launch_tables(const DeviceModel& m, const float* params, const uint8_t* pixels,
                          long long n, uint32_t* cum, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  tables_kernel<<<grid_for(n, kWarps, 4096), kThreads, 0, s>>>(m.d.K, m.d.NO, params, pixels, n,
                                                               cum);
  return cudaGetLastError();
}

__global__ void rans_enc_test_kernel(const uint32_t* __restrict__ start,
                                     const uint32_t* __restrict__ freq,
                                     const long long* __restrict__ sym_off, int n_streams,
                                     uint8_t* __restrict__ out, long long stride,
                                     int32_t* __restrict__ lens) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_streams) return;
  const long long a = sym_off[s], nsym = sym_off[s + 1] - a;
  lens[s] = rans_encode_stream(
      [&](long long k) { return start[a + k] | (freq[a + k] << 16); }, nsym,
      out + (long long)s * stride + stride);
}

cudaError_t launch_rans_encode(const uint32_t* start, const uint32_t* freq,
                               const long long* sym_off, int n_streams, uint8_t* out,
                               long long stride, int32_t* lens, cudaStream_t s) {
  if (n_streams == 0) return cudaSuccess;
  rans_enc_test_kernel<<<grid_for(n_streams, 128, 1 << 20), 128, 0, s>>>(start, freq, sym_off,
                                                                         n_streams, out, stride,
                                                                         lens);
  return cudaGetLastError();
}

__global__ void rans_dec_test_kernel(const uint8_t* __restrict__ in, long long stride,
                                     const int32_t* __restrict__ lens,
                                     const uint32_t* __restrict__ cum,
                                     const long long* __restrict__ sym_off, int n_streams,
                                     int32_t* __restrict__ sym, int* status) {
  __shared__ TableScratch ws[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int s = blockIdx.x * kWarps + warp;
  if (s >= n_streams) return;
  long long len = lens[s];
  const bool fits = len >= 4 && len <= stride;
  if (!fits) len = 0;
  const uint8_t* base = in + (long long)s * stride + stride - len;
  GroupRansDec dec;
  dec.bad = !fits;
  dec.x = kRansL;
  unsigned long long pos = 4;
  const unsigned long long end = (unsigned long long)len;
  if (!dec.bad)
    dec.x = ((uint32_t)base[0] << 24) | ((uint32_t)base[1] << 16) | ((uint32_t)base[2] << 8) |
            (uint32_t)base[3];
  for (long long k = sym_off[s]; k < sym_off[s + 1]; k++) {
    for (int b = lane; b < 256; b += 32) ws[warp].cum[cum_pos<32>(b)] = cum[k * 257 + b];
    __syncwarp();
    dec.load_bytes(base, pos, end);
    const int v = dec.decode_table<32>(ws[warp], lane);
    pos += dec.used;
    if (lane == 0) sym[k] = v;
    __syncwarp();
  }
  if (lane == 0 && (dec.bad || dec.x != kRansL || pos != end)) set_status(status, ST_CORRUPT);
}

cudaError_t launch_rans_decode(const uint8_t* in, long long stride, const int32_t* lens,
                               const uint32_t* cum, const long long* sym_off, int n_streams,
                               int32_t* sym, int* status, cudaStream_t s) {
  if (n_streams == 0) return cudaSuccess;
  rans_dec_test_kernel<<<grid_for(n_streams, kWarps, 1 << 20), kThreads, 0, s>>>(
      in, stride, lens, cum, sym_off, n_streams, sym, status);
  return cudaGetLastError();
}

}  // namespace nlc

namespace nlc {

// ---------------------------------------------------------------------
// Device check behind the pointwise CDF: ex2.approx must be non-decreasing
// over all floats (-inf .. +inf) and rcp.approx non-increasing on [1, +inf].
// Every pair of adjacent floats in those ranges is compared (5.4e9 pairs,
// a few milliseconds); viol receives the number of pairs out of order.
// ---------------------------------------------------------------------
__global__ void mono_check_kernel(unsigned long long* viol) {
  constexpr uint32_t kInf = 0x7F800000u;  // bit pattern of +inf
  constexpr uint32_t kOne = 0x3F800000u;
  // ranges of bit patterns b, each compared with b + 1:
  //   [0, kInf): x = +0 .. +inf, ex2 non-decreasing
  //   [kInf, 2 kInf): x = -0 .. -inf (value falls as bits rise), ex2 non-increasing
  //   [2 kInf, 2 kInf + kInf - kOne): x = 1 .. +inf, rcp non-increasing
  const unsigned long long n = 2ull * kInf + (kInf - kOne);
  unsigned long long bad = 0;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    if (i < kInf) {
      const uint32_t b = (uint32_t)i;
      bad += ex2_approx(__uint_as_float(b + 1)) < ex2_approx(__uint_as_float(b)) ? 1 : 0;
    } else if (i < 2ull * kInf) {
      const uint32_t b = 0x80000000u | (uint32_t)(i - kInf);
      bad += ex2_approx(__uint_as_float(b + 1)) > ex2_approx(__uint_as_float(b)) ? 1 : 0;
    } else {
      const uint32_t b = kOne + (uint32_t)(i - 2ull * kInf);
      bad += rcp_approx(__uint_as_float(b + 1)) > rcp_approx(__uint_as_float(b)) ? 1 : 0;
    }
  }
  if (bad) atomicAdd(viol, bad);
}

cudaError_t launch_mono_check(unsigned long long* viol, int sm_count, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(viol, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  mono_check_kernel<<<sm_count * 8, 256, 0, s>>>(viol);
  return cudaGetLastError();
}

}  // namespace nlc
