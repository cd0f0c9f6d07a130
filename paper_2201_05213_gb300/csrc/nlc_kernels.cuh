// Host-visible declarations of the kernels' launchers (internal to the
// library; the public surface is include/nlc.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nlc_common.cuh"

namespace nlc {

// Per-image record of a batch.
struct ImageRec {
  int H, W;
  int stream_base, n_streams;
  int unit_base, n_units;
};

// Container header (32 bytes, little endian), followed by n_streams uint32
// stream lengths in bytes, then the streams back to back; the container is
// zero-padded to a multiple of 16 bytes.
constexpr uint32_t kMagic = 0x31434C4Eu;  // "NLC1"
constexpr int kVersion = 2;
constexpr int kHeaderBytes = 32;

// Bytes per entry of a container's stream-length table: 2 when no stream of
// the image can reach 2^16 bytes (a pixel codes to at most 6 bytes, a
// stream adds 4: 6 px + 4 < 2^16 for the largest stream of the image's
// geometry), else 4.  A function of (H, W, patch, layout) alone, so the
// decoder derives it from the header.
__host__ __device__ __forceinline__ int len_width(int H, int W, int patch, int layout) {
  const long long P = patch > 0 ? patch : (H > W ? H : W);
  const long long w = W < P ? W : P, hh = H < P ? H : P;
  const long long px = layout == 1 ? w : hh * w;
  return 6 * px + 4 < 65536 ? 2 : 4;
}

struct DeviceModel {
  Dims d;
  WeightView w;
  const unsigned long long* hash;
};

// Decoder state of one rANS stream between wavefront steps: state x, the
// next 8 stream bytes (b0 = bytes pos .. pos+3, little-endian; b1 = pos+4 ..
// pos+7; bytes at or past `end` are unspecified and never consumed by a
// valid stream), the read position and the end (absolute offsets into the
// batch of containers).  Copied to shared memory with two 16-byte cp.async.
struct alignas(16) StreamRec {
  uint32_t x, b0, b1, pad;
  unsigned long long pos, end;
};

// Per-call device buffers (sub-allocated from the context workspace).
struct CodecBufs {
  const Unit* units;
  const ImageRec* images;
  int n_units, n_images, n_streams;
  long long n_px;
  // encoder
  uint32_t* stage;               // 3 * n_px packed (start | freq << 16)
  uint8_t* scratch;              // per-stream byte slots
  int32_t* lens;                 // n_streams
  unsigned long long* unit_bytes;  // n_units
  unsigned long long* unit_off;    // n_units (absolute byte offset of the unit's first stream)
  // encoder scratch (u64 per stream)
  unsigned long long* st_pos;
  // decoder
  StreamRec* st;
  uint8_t* ring = nullptr;       // sheared wavefront decoder: 96 bytes per unit row
  unsigned* bar;                 // 2 words: arrivals, generation
  int* status;
  unsigned long long* prof = nullptr;  // decoder phase cycle counters (16), optional
  unsigned long long* times = nullptr;  // decoder step end times, optional
  long long n_times = 0;
  unsigned spin_limit = 0;  // decoder: polls of the grid barrier / an MMA completion before a
  unsigned mma_limit = 0;   // timeout is recorded (0: the defaults)
};

// Launchers (return cudaError_t of the launch).
// hash == nullptr: the packed copies only (the content hash is left as is)
cudaError_t launch_repack(const Dims& d, const float* w, float* simt, uint16_t* umma, float* bias,
                          unsigned long long* hash, int n_w, cudaStream_t s);
cudaError_t launch_hash(const Dims& d, const float* w, int n_w, unsigned long long* hash,
                        cudaStream_t s);

cudaError_t launch_encode(const DeviceModel& m, const CodecBufs& b, int layout, int patch,
                          uint8_t* out, unsigned long long cap, unsigned long long* d_offsets,
                          int sm_count, cudaStream_t s);
cudaError_t launch_enc_tables(const DeviceModel& m, const CodecBufs& b, int sm_count,
                              cudaStream_t s);
cudaError_t launch_parse(const DeviceModel& m, const CodecBufs& b, const uint8_t* in,
                         const unsigned long long* d_offsets, int layout, int patch,
                         cudaStream_t s);
// set_attr = false skips cudaFuncSetAttribute (already set by decode_max_grid
// for the same batch), so that the call issues device work only.
cudaError_t launch_decode(const DeviceModel& m, const CodecBufs& b, const uint8_t* in,
                          const unsigned long long* d_offsets, int layout, int patch, int sched,
                          int T, int grid, cudaStream_t s, bool set_attr = true);
// win: the sheared model's wavefront decoder (window tiles from the ring).
int decode_max_grid(const DeviceModel& m, int n_units, int sm_count, bool sample = false,
                    bool win = false);
// The decoder's schedule and tables driven by a counter-based generator
// instead of streams: draws the batch's pixels from the model.
cudaError_t launch_sample(const DeviceModel& m, const CodecBufs& b, int sched, int T, int grid,
                          unsigned long long seed, cudaStream_t s);
size_t decode_smem_bytes(const Dims& d, int n_units);
cudaError_t launch_forward(const DeviceModel& m, const CodecBufs& b, float* params, float* bits,
                           int sm_count, cudaStream_t s);
cudaError_t launch_tables(const DeviceModel& m, const float* params, const uint8_t* pixels,
                          long long n, uint32_t* cum, cudaStream_t s);
cudaError_t launch_rans_encode(const uint32_t* start, const uint32_t* freq,
                               const long long* sym_off, int n_streams, uint8_t* out,
                               long long stride, int32_t* lens, cudaStream_t s);
cudaError_t launch_rans_decode(const uint8_t* in, long long stride, const int32_t* lens,
                               const uint32_t* cum, const long long* sym_off, int n_streams,
                               int32_t* sym, int* status, cudaStream_t s);
// Counts adjacent float pairs on which ex2.approx / rcp.approx are not
// monotone over the ranges the frequency tables use (0 expected).
cudaError_t launch_mono_check(unsigned long long* viol, int sm_count, cudaStream_t s);

}  // namespace nlc
