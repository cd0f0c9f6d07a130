// Host side of the nlc C ABI (include/nlc.h): argument validation, the
// context (weights, optimizer state, device workspace), batch planning
// (coding units, streams, schedules) and kernel launches.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "../../include/nlc.h"
#include "nlc_common.cuh"
#include "nlc_kernels.cuh"
#include "nlc_model.cuh"
#include "nlc_tc.cuh"
#include "nlc_train.cuh"

using namespace nlc;

static thread_local char g_err[512] = "no error";

static int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

#define CUDA_TRY(x)                                                                  \
  do {                                                                               \
    cudaError_t e_ = (x);                                                            \
    if (e_ != cudaSuccess)                                                           \
      return fail(NLC_ERR_CUDA, "%s failed: %s", #x, cudaGetErrorString(e_));        \
  } while (0)

struct nlc_ctx {
  Dims d;
  int device = 0, sm_count = 0;
  size_t n_w = 0;
  float* d_w = nullptr;
  float* d_simt = nullptr;
  uint16_t* d_umma = nullptr;
  float* d_bias = nullptr;
  unsigned long long* d_hash = nullptr;
  int* d_status = nullptr;
  float* d_m = nullptr;  // Adam moments
  float* d_v = nullptr;
  float* d_grad = nullptr;
  float* d_loss = nullptr;
  long long adam_t = 0;
  bool dirty = true;       // packed weight copies out of date
  bool hash_dirty = true;  // content hash out of date
  unsigned char* ws = nullptr;
  size_t ws_cap = 0;
  int px_per_cta = 8;
  int max_ctas = 0;
  unsigned long long* d_prof = nullptr;  // decoder phase counters (16), allocated once
  bool prof_on = false;                  // launches receive d_prof only while profiling
  unsigned long long* d_times = nullptr;  // caller's buffer of decoder step end times
  long long n_times = 0;
  unsigned spin_limit = 0, mma_limit = 0;  // decoder wait limits (0: defaults)
};

static unsigned long long* prof_ptr(const nlc_ctx* x) { return x->prof_on ? x->d_prof : nullptr; }

extern "C" const char* nlc_last_error(void) { return g_err; }
extern "C" int nlc_abi_version(void) { return NLC_ABI_VERSION; }

static bool cfg_ok(const nlc_model_cfg* c) {
  return c && c->h >= 1 && c->h <= kMaxH && (c->C == 16 || c->C == 32 || c->C == 48 ||
                                               c->C == 64) &&
         c->n_res >= 0 && c->n_res <= kMaxR && c->K >= 1 && c->K <= kMaxK &&
         (c->precision == NLC_FP32 || c->precision == NLC_BF16 ||
          c->precision == NLC_BF16_SHEARED);
}

static Dims make_dims(const nlc_model_cfg* c) {
  Dims d;
  d.h = c->h;
  d.C = c->C;
  d.R = c->n_res;
  d.K = c->K;
  d.F = 6 * c->h * (c->h + 1);
  d.Fp = (d.F + 15) / 16 * 16;
  d.NO = 10 * c->K;
  d.NOp = (d.NO + 15) / 16 * 16;
  d.ldP = d.NOp + 1;  // odd: one pixel per lane stores its row without bank conflicts
  d.shear = c->precision == NLC_BF16_SHEARED ? 1 : 0;
  d.prec = d.shear ? NLC_BF16 : c->precision;
  d.Ws = c->h * (c->h + 2);
  d.Fsp = shear_row_features_n(c->h);  // 16, 32, 56 for h = 1, 2, 3
  return d;
}

extern "C" size_t nlc_num_weights(const nlc_model_cfg* c) {
  if (!cfg_ok(c)) return 0;
  const size_t F = 6 * c->h * (c->h + 1), C = c->C;
  return C * F + C + (size_t)c->n_res * 2 * (C * C + C) + 10 * (size_t)c->K * C + 10 * (size_t)c->K;
}

static DeviceModel model_view(const nlc_ctx* x) {
  DeviceModel m;
  m.d = x->d;
  m.w.simt = x->d_simt;
  m.w.umma = x->d_umma;
  m.w.bias = x->d_bias;
  m.w.simt_floats = (int)simt_floats(x->d);
  m.w.umma_halves = (int)umma_halves(x->d);
  m.hash = x->d_hash;
  return m;
}

// Brings the packed weight copies (and, with hash, the content hash that the
// containers carry) up to date.  Training steps skip the hash: only the
// codec calls need it.
static int ensure_packed(nlc_ctx* x, cudaStream_t s, bool hash = true) {
  if (x->dirty) {
    CUDA_TRY(launch_repack(x->d, x->d_w, x->d_simt, x->d_umma, x->d_bias, nullptr, (int)x->n_w, s));
    x->dirty = false;
    x->hash_dirty = true;
  }
  if (hash && x->hash_dirty) {
    CUDA_TRY(launch_hash(x->d, x->d_w, (int)x->n_w, x->d_hash, s));
    x->hash_dirty = false;
  }
  return NLC_OK;
}

extern "C" int nlc_destroy(nlc_ctx* x) {
  if (!x) return NLC_OK;
  cudaDeviceSynchronize();
  cudaFree(x->d_w);
  cudaFree(x->d_simt);
  cudaFree(x->d_umma);
  cudaFree(x->d_bias);
  cudaFree(x->d_hash);
  cudaFree(x->d_status);
  cudaFree(x->d_m);
  cudaFree(x->d_v);
  cudaFree(x->d_grad);
  cudaFree(x->d_loss);
  cudaFree(x->d_prof);
  cudaFree(x->ws);
  delete x;
  return NLC_OK;
}

// Result of the monotonicity check of the MUFU approximations per device
// (0 = not run, 1 = passed, -1 = failed), run once per device and process.
static std::mutex g_mono_mu;
static int g_mono[64];

static int check_mono(int device, int sm_count, unsigned long long* d_scratch) {
  std::lock_guard<std::mutex> lock(g_mono_mu);
  const int slot = device >= 0 && device < 64 ? device : 63;
  if (g_mono[slot] == 0) {
    cudaError_t e = launch_mono_check(d_scratch, sm_count, 0);
    unsigned long long viol = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&viol, d_scratch, 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(NLC_ERR_CUDA, "device check failed: %s", cudaGetErrorString(e));
    g_mono[slot] = viol == 0 ? 1 : -1;
  }
  if (g_mono[slot] < 0)
    return fail(NLC_ERR_UNSUPPORTED,
                "ex2.approx / rcp.approx are not monotone on this device; the frequency tables "
                "need them to be");
  return NLC_OK;
}

extern "C" int nlc_create(const nlc_model_cfg* cfg, const float* h_w, size_t n, nlc_ctx** out) {
  if (!out) return fail(NLC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!cfg_ok(cfg))
    return fail(NLC_ERR_UNSUPPORTED,
                "unsupported configuration (h 1..3, C in {16,32,48,64}, n_res 0..4, K 1..16, "
                "precision 0/1/2)");
  if (!h_w || n != nlc_num_weights(cfg))
    return fail(NLC_ERR_ARG, "expected %zu weights, got %zu", nlc_num_weights(cfg), n);
  nlc_ctx* x = new nlc_ctx();
  x->d = make_dims(cfg);
  x->n_w = n;
  int rc = NLC_OK;
  do {
    cudaError_t e;
#define TRY_ALLOC(p, bytes)                                                             \
  if ((e = cudaMalloc((void**)&(p), (bytes))) != cudaSuccess) {                         \
    rc = fail(NLC_ERR_CUDA, "cudaMalloc failed: %s", cudaGetErrorString(e));            \
    break;                                                                              \
  }
    if ((e = cudaGetDevice(&x->device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&x->sm_count, cudaDevAttrMultiProcessorCount, x->device)) !=
            cudaSuccess) {
      rc = fail(NLC_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
      break;
    }
    TRY_ALLOC(x->d_w, n * 4);
    TRY_ALLOC(x->d_simt, simt_floats(x->d) * 4);
    TRY_ALLOC(x->d_umma, umma_halves(x->d) * 2);
    TRY_ALLOC(x->d_bias, bias_floats(x->d) * 4);
    TRY_ALLOC(x->d_hash, 8);
    TRY_ALLOC(x->d_status, 4);
    TRY_ALLOC(x->d_m, n * 4);
    TRY_ALLOC(x->d_v, n * 4);
    TRY_ALLOC(x->d_grad, n * 4);
    TRY_ALLOC(x->d_loss, 8);
    TRY_ALLOC(x->d_prof, 16 * sizeof(uint64_t));
    if ((e = cudaMemset(x->d_prof, 0, 16 * sizeof(uint64_t))) != cudaSuccess) {
      rc = fail(NLC_ERR_CUDA, "initialisation failed: %s", cudaGetErrorString(e));
      break;
    }
    rc = check_mono(x->device, x->sm_count, reinterpret_cast<unsigned long long*>(x->d_loss));
    if (rc) break;
    if ((e = cudaMemcpy(x->d_w, h_w, n * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(x->d_status, 0, 4)) != cudaSuccess ||
        (e = cudaMemset(x->d_m, 0, n * 4)) != cudaSuccess ||
        (e = cudaMemset(x->d_v, 0, n * 4)) != cudaSuccess) {
      rc = fail(NLC_ERR_CUDA, "initialisation failed: %s", cudaGetErrorString(e));
      break;
    }
    rc = ensure_packed(x, 0);
    if (rc) break;
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
      rc = fail(NLC_ERR_CUDA, "weight packing failed: %s", cudaGetErrorString(e));
      break;
    }
#undef TRY_ALLOC
  } while (0);
  if (rc != NLC_OK) {
    nlc_destroy(x);
    return rc;
  }
  *out = x;
  return NLC_OK;
}

extern "C" int nlc_get_weights(nlc_ctx* x, float* h_w, size_t n) {
  if (!x || !h_w || n != x->n_w) return fail(NLC_ERR_ARG, "bad arguments");
  CUDA_TRY(cudaDeviceSynchronize());
  CUDA_TRY(cudaMemcpy(h_w, x->d_w, n * 4, cudaMemcpyDeviceToHost));
  return NLC_OK;
}

extern "C" int nlc_set_weights(nlc_ctx* x, const float* h_w, size_t n) {
  if (!x || !h_w || n != x->n_w) return fail(NLC_ERR_ARG, "bad arguments");
  CUDA_TRY(cudaDeviceSynchronize());
  CUDA_TRY(cudaMemcpy(x->d_w, h_w, n * 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemset(x->d_m, 0, n * 4));
  CUDA_TRY(cudaMemset(x->d_v, 0, n * 4));
  x->adam_t = 0;
  x->dirty = true;
  int rc = ensure_packed(x, 0);
  if (rc) return rc;
  CUDA_TRY(cudaDeviceSynchronize());
  return NLC_OK;
}

extern "C" int nlc_weight_hash(nlc_ctx* x, uint64_t* h) {
  if (!x || !h) return fail(NLC_ERR_ARG, "bad arguments");
  int rc = ensure_packed(x, 0);
  if (rc) return rc;
  CUDA_TRY(cudaDeviceSynchronize());
  CUDA_TRY(cudaMemcpy(h, x->d_hash, 8, cudaMemcpyDeviceToHost));
  return NLC_OK;
}

extern "C" int nlc_sync_status(nlc_ctx* x, nlc_stream stream) {
  if (!x) return fail(NLC_ERR_ARG, "ctx is NULL");
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  int st = 0;
  CUDA_TRY(cudaMemcpy(&st, x->d_status, 4, cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemset(x->d_status, 0, 4));
  switch (st) {
    case 0: return NLC_OK;
    case ST_CAPACITY: return fail(NLC_ERR_CAPACITY, "output capacity exceeded");
    case ST_CORRUPT: return fail(NLC_ERR_CORRUPT, "corrupt container or stream");
    case ST_WEIGHTS: return fail(NLC_ERR_WEIGHTS, "container made with other weights or precision");
    case ST_TIMEOUT: return fail(NLC_ERR_TIMEOUT, "a bounded device wait timed out");
    default: return fail(st, "device status %d", st);
  }
}

extern "C" int nlc_decode_step_times(nlc_ctx* x, uint64_t* d_times, int64_t n) {
  if (!x || n < 0 || (n > 0 && !d_times)) return fail(NLC_ERR_ARG, "bad arguments");
  if (reinterpret_cast<uintptr_t>(d_times) % 8) return fail(NLC_ERR_ARG, "d_times must be 8-byte aligned");
  x->d_times = n > 0 ? reinterpret_cast<unsigned long long*>(d_times) : nullptr;
  x->n_times = n;
  return NLC_OK;
}

extern "C" int nlc_decode_profile(nlc_ctx* x, int enable, uint64_t* h_counters) {
  if (!x) return fail(NLC_ERR_ARG, "ctx is NULL");
  CUDA_TRY(cudaDeviceSynchronize());
  if (h_counters)
    CUDA_TRY(cudaMemcpy(h_counters, x->d_prof, 16 * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  if (h_counters || enable != (int)x->prof_on)
    CUDA_TRY(cudaMemset(x->d_prof, 0, 16 * sizeof(uint64_t)));
  x->prof_on = enable != 0;
  return NLC_OK;
}

extern "C" int nlc_set_wait_limits(nlc_ctx* x, uint32_t grid_polls, uint32_t mma_polls) {
  if (!x) return fail(NLC_ERR_ARG, "ctx is NULL");
  x->spin_limit = grid_polls;
  x->mma_limit = mma_polls;
  return NLC_OK;
}

extern "C" int nlc_set_tuning(nlc_ctx* x, int px_per_cta, int max_ctas) {
  if (!x || px_per_cta < 1 || max_ctas < 0) return fail(NLC_ERR_ARG, "bad arguments");
  x->px_per_cta = px_per_cta;
  x->max_ctas = max_ctas;
  return NLC_OK;
}

// ---------------------------------------------------------------------
// Batch planning
// ---------------------------------------------------------------------
struct Batch {
  std::vector<Unit> units;
  std::vector<ImageRec> images;
  long long n_px = 0;
  int n_streams = 0;
  long long T = 0;        // decode steps
  long long max_front = 0;
  long long ring_rows = 0;  // rows of all units (the sheared decoder's ring)
};

static int plan_batch(const Dims& d, int n, uint8_t* const* ptrs, const int32_t* H,
                      const int32_t* W, int patch, int layout, int sched_mode, Batch& b) {
  b.units.clear();
  b.images.clear();
  b.n_px = 0;
  b.n_streams = 0;
  b.T = 0;
  b.max_front = 0;
  const int o = d.h + 1;
  int ring_rows = 0;
  for (int i = 0; i < n; i++) {
    const long long img_px_base = b.n_px;
    ImageRec I;
    I.H = H[i];
    I.W = W[i];
    I.stream_base = b.n_streams;
    I.unit_base = (int)b.units.size();
    I.n_units = 0;
    long long img_start = 0;
    const bool empty = H[i] == 0 || W[i] == 0;
    const int P = patch > 0 ? patch : std::max(H[i], W[i]);
    if (!empty) {
      for (int y = 0; y < H[i]; y += P)
        for (int xx = 0; xx < W[i]; xx += P) {
          Unit u;
          u.img = ptrs[i];
          u.px_base = b.n_px;
          u.img_W = W[i];
          u.y0 = y;
          u.x0 = xx;
          u.Hu = std::min(P, H[i] - y);
          u.Wu = std::min(P, W[i] - xx);
          u.stream_base = b.n_streams;
          u.image = i;
          u.ring_row = ring_rows;
          ring_rows += u.Hu;
          u.img_px_base = img_px_base;
          long long Tu;
          if (sched_mode == NLC_SCHED_WAVEFRONT) {
            u.start_step = 0;
            Tu = u.Wu + (long long)(u.Hu - 1) * o;
            b.max_front += std::min<long long>(u.Hu, (u.Wu + o - 1) / o);
          } else if (sched_mode == NLC_SCHED_RASTER) {
            u.start_step = 0;
            Tu = (long long)u.Hu * u.Wu;
            b.max_front += 1;
          } else {
            if (img_start > INT32_MAX) return fail(NLC_ERR_UNSUPPORTED, "image too large");
            u.start_step = (int)img_start;
            Tu = (long long)u.Hu * u.Wu;
            img_start += Tu;
          }
          b.T = std::max(b.T, (long long)u.start_step + Tu);
          b.n_px += (long long)u.Hu * u.Wu;
          b.n_streams += layout == NLC_LAYOUT_ROW ? u.Hu : 1;
          b.units.push_back(u);
          I.n_units++;
        }
      if (sched_mode == NLC_SCHED_SEQUENTIAL) b.max_front += 1;
    }
    I.n_streams = b.n_streams - I.stream_base;
    b.images.push_back(I);
  }
  b.ring_rows = ring_rows;
  if (b.T > INT32_MAX || b.n_px > (1LL << 40))
    return fail(NLC_ERR_UNSUPPORTED, "batch too large");
  return NLC_OK;
}

static int check_images(int n, const int32_t* H, const int32_t* W, const void* const* data,
                        int patch) {
  if (n < 0) return fail(NLC_ERR_ARG, "n < 0");
  if (patch < 0) return fail(NLC_ERR_ARG, "patch < 0");
  for (int i = 0; i < n; i++) {
    if (H[i] < 0 || W[i] < 0) return fail(NLC_ERR_ARG, "image %d has a negative size", i);
    if ((long long)H[i] * W[i] > 0 && !data[i])
      return fail(NLC_ERR_ARG, "image %d has no data pointer", i);
    if ((long long)H[i] * W[i] > (1LL << 31)) return fail(NLC_ERR_UNSUPPORTED, "image too large");
  }
  return NLC_OK;
}

// Workspace arena (256-byte aligned pieces).
struct Arena {
  unsigned char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += (count * sizeof(T) + 255) & ~(size_t)255;
    return p;
  }
};

static int ensure_ws(nlc_ctx* x, size_t bytes) {
  if (bytes <= x->ws_cap) return NLC_OK;
  CUDA_TRY(cudaDeviceSynchronize());
  cudaFree(x->ws);
  x->ws = nullptr;
  x->ws_cap = 0;
  size_t cap = std::max(bytes, x->ws_cap * 2);
  CUDA_TRY(cudaMalloc((void**)&x->ws, cap));
  x->ws_cap = cap;
  return NLC_OK;
}

// Lays out the per-call buffers; with base == nullptr only measures.
static size_t layout_bufs(const Batch& b, unsigned char* base, CodecBufs& cb, int* status,
                          bool encode, bool ring = false) {
  Arena a{base};
  const size_t U = b.units.size(), S = (size_t)b.n_streams;
  cb.units = a.take<Unit>(U + 1);
  cb.images = a.take<ImageRec>(b.images.size() + 1);
  cb.n_units = (int)U;
  cb.n_images = (int)b.images.size();
  cb.n_streams = (int)S;
  cb.n_px = b.n_px;
  cb.lens = a.take<int32_t>(S + 1);
  cb.unit_bytes = a.take<unsigned long long>(U + 1 + (b.images.size() + 1) / 2 + 1);
  cb.unit_off = a.take<unsigned long long>(U + 1);
  cb.st_pos = a.take<unsigned long long>(S + 1);
  cb.st = a.take<StreamRec>(S + 1);
  cb.bar = a.take<unsigned>(64);
  if (encode) {
    cb.stage = a.take<uint32_t>(3 * (size_t)b.n_px + 1);
    cb.scratch = a.take<uint8_t>(6 * (size_t)b.n_px + 4 * S + 16);
  } else {
    cb.stage = nullptr;
    cb.scratch = nullptr;
  }
  cb.ring = ring ? a.take<uint8_t>((size_t)kRingRowBytes * (size_t)(b.ring_rows + 1)) : nullptr;
  cb.status = status;
  return a.off;
}

static int upload_batch(const Batch& b, CodecBufs& cb, cudaStream_t s) {
  if (!b.units.empty())
    CUDA_TRY(cudaMemcpyAsync((void*)cb.units, b.units.data(), b.units.size() * sizeof(Unit),
                             cudaMemcpyHostToDevice, s));
  if (!b.images.empty())
    CUDA_TRY(cudaMemcpyAsync((void*)cb.images, b.images.data(), b.images.size() * sizeof(ImageRec),
                             cudaMemcpyHostToDevice, s));
  return NLC_OK;
}

extern "C" int nlc_compress_bound(const int32_t* H, const int32_t* W, int n, int patch, int layout,
                                  size_t* bytes) {
  if (!bytes || (n > 0 && (!H || !W)) || n < 0 || patch < 0 || (layout != 0 && layout != 1))
    return fail(NLC_ERR_ARG, "bad arguments");
  size_t tot = 0;
  for (int i = 0; i < n; i++) {
    if (H[i] < 0 || W[i] < 0) return fail(NLC_ERR_ARG, "negative image size");
    size_t ns = 0;
    if (H[i] > 0 && W[i] > 0) {
      const int P = patch > 0 ? patch : std::max(H[i], W[i]);
      const size_t nu = (size_t)((H[i] + P - 1) / P) * ((W[i] + P - 1) / P);
      ns = layout == 1 ? (size_t)((W[i] + P - 1) / P) * H[i] : nu;
    }
    size_t c = kHeaderBytes + 8 * ns + 6 * (size_t)H[i] * W[i];
    tot += (c + 15) & ~(size_t)15;
  }
  *bytes = tot;
  return NLC_OK;
}

extern "C" int nlc_compress(nlc_ctx* x, const nlc_image_in* imgs, int n, int patch, int layout,
                            uint8_t* d_out, size_t cap, uint64_t* d_offsets, nlc_stream stream) {
  if (!x || n < 0 || (n > 0 && !imgs) || !d_offsets || (layout != 0 && layout != 1))
    return fail(NLC_ERR_ARG, "bad arguments");
  std::vector<int32_t> H(n), W(n);
  std::vector<const void*> data(n);
  std::vector<uint8_t*> ptrs(n);
  for (int i = 0; i < n; i++) {
    H[i] = imgs[i].H;
    W[i] = imgs[i].W;
    data[i] = imgs[i].data;
    ptrs[i] = const_cast<uint8_t*>(imgs[i].data);
  }
  int rc = check_images(n, H.data(), W.data(), data.data(), patch);
  if (rc) return rc;
  if (!d_out && cap > 0) return fail(NLC_ERR_ARG, "d_out is NULL");
  if (reinterpret_cast<uintptr_t>(d_out) % 16) return fail(NLC_ERR_ARG, "d_out must be 16-byte aligned");
  Batch b;
  rc = plan_batch(x->d, n, ptrs.data(), H.data(), W.data(), patch, layout, NLC_SCHED_RASTER, b);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  CodecBufs cb;
  size_t need = layout_bufs(b, nullptr, cb, x->d_status, true);
  if ((rc = ensure_ws(x, need))) return rc;
  layout_bufs(b, x->ws, cb, x->d_status, true);
  if ((rc = ensure_packed(x, s))) return rc;
  if ((rc = upload_batch(b, cb, s))) return rc;
  CUDA_TRY(launch_encode(model_view(x), cb, layout, patch, d_out, (unsigned long long)cap,
                         reinterpret_cast<unsigned long long*>(d_offsets), x->sm_count, s));
  return NLC_OK;
}

extern "C" int nlc_decompress(nlc_ctx* x, const uint8_t* d_in, const uint64_t* d_offsets,
                              const nlc_image_out* outs, int n, int patch, int layout,
                              int schedule, nlc_stream stream) {
  if (!x || n < 0 || (n > 0 && (!outs || !d_in || !d_offsets)) || (layout != 0 && layout != 1))
    return fail(NLC_ERR_ARG, "bad arguments");
  if (schedule < 0 || schedule > 2) return fail(NLC_ERR_ARG, "unknown schedule %d", schedule);
  if (reinterpret_cast<uintptr_t>(d_in) % 16) return fail(NLC_ERR_ARG, "d_in must be 16-byte aligned");
  if (layout == NLC_LAYOUT_UNIT && schedule == NLC_SCHED_WAVEFRONT)
    return fail(NLC_ERR_ARG, "one stream per unit can only be decoded in raster order");
  std::vector<int32_t> H(n), W(n);
  std::vector<const void*> data(n);
  std::vector<uint8_t*> ptrs(n);
  for (int i = 0; i < n; i++) {
    H[i] = outs[i].H;
    W[i] = outs[i].W;
    data[i] = outs[i].data;
    ptrs[i] = outs[i].data;
  }
  int rc = check_images(n, H.data(), W.data(), data.data(), patch);
  if (rc) return rc;
  Batch b;
  rc = plan_batch(x->d, n, ptrs.data(), H.data(), W.data(), patch, layout, schedule, b);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const DeviceModel m = model_view(x);
  if (decode_smem_bytes(x->d, (int)b.units.size()) > 227 * 1024)
    return fail(NLC_ERR_UNSUPPORTED, "too many coding units in one call (%zu)", b.units.size());
  CodecBufs cb;
  const bool ring = x->d.shear && schedule == NLC_SCHED_WAVEFRONT;
  if (ring && b.ring_rows >= (1LL << 31) / kRingRowBytes)
    return fail(NLC_ERR_UNSUPPORTED, "batch too large for the sheared decoder's rings");
  size_t need = layout_bufs(b, nullptr, cb, x->d_status, false, ring);
  if ((rc = ensure_ws(x, need))) return rc;
  layout_bufs(b, x->ws, cb, x->d_status, false, ring);
  if ((rc = ensure_packed(x, s))) return rc;
  if ((rc = upload_batch(b, cb, s))) return rc;
  int gmax = decode_max_grid(m, (int)b.units.size(), x->sm_count, false, ring);
  if (gmax < 1) return fail(NLC_ERR_UNSUPPORTED, "decoder does not fit on an SM");
  if (x->max_ctas > 0) gmax = std::min(gmax, x->max_ctas);
  long long g = (b.max_front + x->px_per_cta - 1) / x->px_per_cta;
  int grid = (int)std::max(1LL, std::min<long long>(g, gmax));
  // the barrier's arrival counter reaches grid * T; keep it below 2^31 (bit 31 flags a timeout)
  if ((long long)grid * b.T >= (1LL << 31) - 1) grid = 1;
  const int sched = schedule == NLC_SCHED_WAVEFRONT ? SCHED_WAVEFRONT : SCHED_RASTER;
  cb.prof = prof_ptr(x);
  cb.times = x->d_times;
  cb.n_times = x->n_times;
  cb.spin_limit = x->spin_limit;
  cb.mma_limit = x->mma_limit;
  CUDA_TRY(launch_decode(m, cb, d_in, reinterpret_cast<const unsigned long long*>(d_offsets),
                         layout, patch, sched, (int)b.T, grid, s));
  return NLC_OK;
}

extern "C" int nlc_sample(nlc_ctx* x, const nlc_image_out* outs, int n, int patch,
                          uint64_t seed, int schedule, nlc_stream stream) {
  if (!x || n < 0 || (n > 0 && !outs)) return fail(NLC_ERR_ARG, "bad arguments");
  if (schedule < 0 || schedule > 2) return fail(NLC_ERR_ARG, "unknown schedule %d", schedule);
  std::vector<int32_t> H(n), W(n);
  std::vector<const void*> data(n);
  std::vector<uint8_t*> ptrs(n);
  for (int i = 0; i < n; i++) {
    H[i] = outs[i].H;
    W[i] = outs[i].W;
    data[i] = outs[i].data;
    ptrs[i] = outs[i].data;
  }
  int rc = check_images(n, H.data(), W.data(), data.data(), patch);
  if (rc) return rc;
  for (int i = 0; i < n; i++)
    if (H[i] >= (1 << 21) || W[i] >= (1 << 21) || i >= (1 << 21))
      return fail(NLC_ERR_UNSUPPORTED, "the sampler's counter needs sides and n below 2^21");
  Batch b;
  rc = plan_batch(x->d, n, ptrs.data(), H.data(), W.data(), patch, NLC_LAYOUT_ROW, schedule, b);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const DeviceModel m = model_view(x);
  if (decode_smem_bytes(x->d, (int)b.units.size()) > 227 * 1024)
    return fail(NLC_ERR_UNSUPPORTED, "too many coding units in one call (%zu)", b.units.size());
  CodecBufs cb;
  const bool ring = x->d.shear && schedule == NLC_SCHED_WAVEFRONT;
  if (ring && b.ring_rows >= (1LL << 31) / kRingRowBytes)
    return fail(NLC_ERR_UNSUPPORTED, "batch too large for the sheared decoder's rings");
  size_t need = layout_bufs(b, nullptr, cb, x->d_status, false, ring);
  if ((rc = ensure_ws(x, need))) return rc;
  layout_bufs(b, x->ws, cb, x->d_status, false, ring);
  if ((rc = ensure_packed(x, s))) return rc;
  if ((rc = upload_batch(b, cb, s))) return rc;
  int gmax = decode_max_grid(m, (int)b.units.size(), x->sm_count, true, ring);
  if (gmax < 1) return fail(NLC_ERR_UNSUPPORTED, "sampler does not fit on an SM");
  if (x->max_ctas > 0) gmax = std::min(gmax, x->max_ctas);
  long long g = (b.max_front + x->px_per_cta - 1) / x->px_per_cta;
  int grid = (int)std::max(1LL, std::min<long long>(g, gmax));
  if ((long long)grid * b.T >= (1LL << 31) - 1) grid = 1;
  const int sched = schedule == NLC_SCHED_WAVEFRONT ? SCHED_WAVEFRONT : SCHED_RASTER;
  cb.spin_limit = x->spin_limit;
  cb.mma_limit = x->mma_limit;
  CUDA_TRY(launch_sample(m, cb, sched, (int)b.T, grid, (unsigned long long)seed, s));
  return NLC_OK;
}

extern "C" int nlc_forward(nlc_ctx* x, const nlc_image_in* imgs, int n, int patch, float* d_params,
                           float* d_bits, nlc_stream stream) {
  if (!x || n < 0 || (n > 0 && !imgs)) return fail(NLC_ERR_ARG, "bad arguments");
  std::vector<int32_t> H(n), W(n);
  std::vector<const void*> data(n);
  std::vector<uint8_t*> ptrs(n);
  for (int i = 0; i < n; i++) {
    H[i] = imgs[i].H;
    W[i] = imgs[i].W;
    data[i] = imgs[i].data;
    ptrs[i] = const_cast<uint8_t*>(imgs[i].data);
  }
  int rc = check_images(n, H.data(), W.data(), data.data(), patch);
  if (rc) return rc;
  Batch b;
  rc = plan_batch(x->d, n, ptrs.data(), H.data(), W.data(), patch, 1, NLC_SCHED_RASTER, b);
  if (rc) return rc;
  if (b.n_px > 0 && !d_params && !d_bits) return NLC_OK;
  cudaStream_t s = (cudaStream_t)stream;
  CodecBufs cb;
  size_t need = layout_bufs(b, nullptr, cb, x->d_status, false);
  if ((rc = ensure_ws(x, need))) return rc;
  layout_bufs(b, x->ws, cb, x->d_status, false);
  if ((rc = ensure_packed(x, s))) return rc;
  if ((rc = upload_batch(b, cb, s))) return rc;
  CUDA_TRY(launch_forward(model_view(x), cb, d_params, d_bits, x->sm_count, s));
  return NLC_OK;
}

extern "C" int nlc_tables(nlc_ctx* x, const float* d_params, const uint8_t* d_pixels, int64_t n,
                          uint32_t* d_cum, nlc_stream stream) {
  if (!x || n < 0 || (n > 0 && (!d_params || !d_pixels || !d_cum)))
    return fail(NLC_ERR_ARG, "bad arguments");
  CUDA_TRY(launch_tables(model_view(x), d_params, d_pixels, n, d_cum, (cudaStream_t)stream));
  return NLC_OK;
}

extern "C" int nlc_rans_encode(const uint32_t* d_start, const uint32_t* d_freq,
                               const int64_t* d_sym_off, int n_streams, uint8_t* d_bytes,
                               int64_t stride, int32_t* d_len, nlc_stream stream) {
  if (n_streams < 0 || (n_streams > 0 && (!d_start || !d_freq || !d_sym_off || !d_bytes ||
                                          !d_len || stride < 4)))
    return fail(NLC_ERR_ARG, "bad arguments");
  CUDA_TRY(launch_rans_encode(d_start, d_freq, reinterpret_cast<const long long*>(d_sym_off),
                              n_streams, d_bytes, stride, d_len, (cudaStream_t)stream));
  return NLC_OK;
}

extern "C" int nlc_rans_decode(nlc_ctx* x, const uint8_t* d_bytes, int64_t stride,
                               const int32_t* d_len, const uint32_t* d_cum,
                               const int64_t* d_sym_off, int n_streams, int32_t* d_sym,
                               nlc_stream stream) {
  if (!x || n_streams < 0 ||
      (n_streams > 0 && (!d_bytes || !d_len || !d_cum || !d_sym_off || !d_sym || stride < 4)))
    return fail(NLC_ERR_ARG, "bad arguments");
  CUDA_TRY(launch_rans_decode(d_bytes, stride, d_len, d_cum,
                              reinterpret_cast<const long long*>(d_sym_off), n_streams, d_sym,
                              x->d_status, (cudaStream_t)stream));
  return NLC_OK;
}

// ---------------------------------------------------------------------
// Training
// ---------------------------------------------------------------------
// The adjoint of a batch: BF16 contexts on the tensor cores (when the
// model's tiles fit in a CTA), FP32 contexts (and larger BF16 models) on the
// FP32 SIMT path.  dparams == nullptr: gradient of the mean code length.
static int run_adjoint(nlc_ctx* x, const uint8_t* d_batch, int N, int H, int W,
                       const float* d_dparams, float* d_loss, float* d_grad, cudaStream_t s) {
  const long long npx = (long long)N * H * W;
  if (npx > (1LL << 31) / 16) return fail(NLC_ERR_UNSUPPORTED, "batch too large");
  const bool tc = x->d.prec == NLC_BF16 && tc_train_fits(x->d);  // sheared: the same weights
  if (!tc && !simt_train_fits(x->d))
    return fail(NLC_ERR_UNSUPPORTED, "model too large for the training kernels' shared memory");
  const size_t need = tc ? tc_train_ws_bytes(x->d, npx, x->sm_count)
                         : train_ws_bytes(x->d, npx, x->sm_count);
  int rc = ensure_ws(x, need);
  if (rc) return rc;
  if ((rc = ensure_packed(x, s, false))) return rc;
  if (tc)
    CUDA_TRY(launch_tc_train(x->d, x->d_umma, x->d_bias, d_batch, N, H, W, d_dparams, d_loss,
                             d_grad, x->ws, x->sm_count, x->d_status, s));
  else
    CUDA_TRY(launch_loss_grad(x->d, x->d_w, x->d_simt, d_batch, N, H, W, d_dparams, d_loss,
                              d_grad, x->ws, x->sm_count, s));
  return NLC_OK;
}

extern "C" int nlc_loss_grad(nlc_ctx* x, const uint8_t* d_batch, int N, int H, int W,
                             float* d_loss, float* d_grad, nlc_stream stream) {
  if (!x || N < 1 || H < 1 || W < 1 || !d_batch || !d_loss || !d_grad)
    return fail(NLC_ERR_ARG, "bad arguments");
  return run_adjoint(x, d_batch, N, H, W, nullptr, d_loss, d_grad, (cudaStream_t)stream);
}

extern "C" int nlc_backward(nlc_ctx* x, const uint8_t* d_batch, int N, int H, int W,
                            const float* d_dparams, float* d_dweights, nlc_stream stream) {
  if (!x || N < 1 || H < 1 || W < 1 || !d_batch || !d_dparams || !d_dweights)
    return fail(NLC_ERR_ARG, "bad arguments");
  return run_adjoint(x, d_batch, N, H, W, d_dparams, nullptr, d_dweights, (cudaStream_t)stream);
}

extern "C" int nlc_load_weights(nlc_ctx* x, const float* d_w, size_t n, nlc_stream stream) {
  if (!x || !d_w || n != x->n_w) return fail(NLC_ERR_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(cudaMemcpyAsync(x->d_w, d_w, n * 4, cudaMemcpyDeviceToDevice, s));
  x->dirty = true;
  return ensure_packed(x, s);
}

extern "C" int nlc_train_step(nlc_ctx* x, const uint8_t* d_batch, int N, int H, int W, float lr,
                              float* h_loss, nlc_stream stream) {
  if (!x || N < 1 || H < 1 || W < 1 || !d_batch || !(lr > 0.f))
    return fail(NLC_ERR_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = nlc_loss_grad(x, d_batch, N, H, W, x->d_loss, x->d_grad, stream);
  if (rc) return rc;
  x->adam_t += 1;
  CUDA_TRY(launch_adam(x->d_w, x->d_grad, x->d_m, x->d_v, (int)x->n_w, lr, 0.9f, 0.999f, 1e-8f,
                       x->adam_t, s));
  x->dirty = true;
  if (h_loss) {
    CUDA_TRY(cudaMemcpyAsync(h_loss, x->d_loss, 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  return NLC_OK;
}

// ---------------------------------------------------------------------
// Compression without allocation (nlc_compress_noalloc).
//
// The batch plan, the per-symbol staging tables and the per-stream byte
// slots live in one file-scope device array instead of the context's
// workspace.  Its name is only a host-side stand-in for the device array, so
// host code asks the runtime for the device address once per device (with
// that device current) and passes that pointer to the kernels.  No byte of
// the array needs to start at zero: every call writes each byte it reads
// before reading it.  All calls share the array, so calls that overlap on
// the GPU (on different streams, or from different contexts) race.
// ---------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[NLC_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[256];

static int noalloc_scratch(void** out) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return fail(NLC_ERR_UNSUPPORTED, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(NLC_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed: %s",
                  cudaGetErrorString(e));
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return NLC_OK;
}

extern "C" int nlc_compress_noalloc(nlc_ctx* x, const nlc_image_in* imgs, int n, int patch,
                                    int layout, uint8_t* d_out, size_t cap, uint64_t* d_offsets,
                                    nlc_stream stream) {
  if (!x || n < 0 || (n > 0 && !imgs) || !d_offsets || (layout != 0 && layout != 1))
    return fail(NLC_ERR_ARG, "bad arguments");
  std::vector<int32_t> H(n), W(n);
  std::vector<const void*> data(n);
  std::vector<uint8_t*> ptrs(n);
  for (int i = 0; i < n; i++) {
    H[i] = imgs[i].H;
    W[i] = imgs[i].W;
    data[i] = imgs[i].data;
    ptrs[i] = const_cast<uint8_t*>(imgs[i].data);
  }
  int rc = check_images(n, H.data(), W.data(), data.data(), patch);
  if (rc) return rc;
  if (!d_out && cap > 0) return fail(NLC_ERR_ARG, "d_out is NULL");
  if (reinterpret_cast<uintptr_t>(d_out) % 16) return fail(NLC_ERR_ARG, "d_out must be 16-byte aligned");
  Batch b;
  rc = plan_batch(x->d, n, ptrs.data(), H.data(), W.data(), patch, layout, NLC_SCHED_RASTER, b);
  if (rc) return rc;
  CodecBufs cb;
  const size_t need = layout_bufs(b, nullptr, cb, x->d_status, true);
  if (need > (size_t)NLC_NOALLOC_SCRATCH_BYTES)
    return fail(NLC_ERR_CAPACITY,
                "batch needs %zu bytes of scratch but nlc_compress_noalloc has %zu; split the "
                "batch or use nlc_compress",
                need, (size_t)NLC_NOALLOC_SCRATCH_BYTES);
  void* base = nullptr;
  if ((rc = noalloc_scratch(&base))) return rc;
  layout_bufs(b, static_cast<unsigned char*>(base), cb, x->d_status, true);
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = ensure_packed(x, s))) return rc;
  if ((rc = upload_batch(b, cb, s))) return rc;
  CUDA_TRY(launch_encode(model_view(x), cb, layout, patch, d_out, (unsigned long long)cap,
                         reinterpret_cast<unsigned long long*>(d_offsets), x->sm_count, s));
  return NLC_OK;
}

// ---------------------------------------------------------------------
// Decode plans: the host work of nlc_decompress (unit partition, schedule,
// device unit tables, grid size) done once, so that a run issues device work
// only and can be captured in a CUDA graph; plus a tuner of the decoder's
// pixels per CTA and step.
// ---------------------------------------------------------------------
struct nlc_plan {
  nlc_ctx* x = nullptr;
  int n = 0, patch = 0, layout = 0, sched = 0;
  long long T = 0, max_front = 0;
  int n_units = 0, grid = 1, gmax = 1, px_per_cta = 8;
  unsigned char* d_buf = nullptr;
  CodecBufs cb;
};

static int plan_grid(const nlc_plan* p, int px_per_cta) {
  long long g = (p->max_front + px_per_cta - 1) / px_per_cta;
  int grid = (int)std::max(1LL, std::min<long long>(g, p->gmax));
  if ((long long)grid * p->T >= (1LL << 31) - 1) grid = 1;
  return grid;
}

extern "C" int nlc_plan_decode(nlc_ctx* x, const nlc_image_out* outs, int n, int patch,
                               int layout, int schedule, nlc_plan** out) {
  if (!out) return fail(NLC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!x || (n > 0 && !outs) || n < 0 || (layout != 0 && layout != 1))
    return fail(NLC_ERR_ARG, "bad arguments");
  if (schedule < 0 || schedule > 2) return fail(NLC_ERR_ARG, "unknown schedule %d", schedule);
  if (layout == NLC_LAYOUT_UNIT && schedule == NLC_SCHED_WAVEFRONT)
    return fail(NLC_ERR_ARG, "one stream per unit can only be decoded in raster order");
  std::vector<int32_t> H(n), W(n);
  std::vector<const void*> data(n);
  std::vector<uint8_t*> ptrs(n);
  for (int i = 0; i < n; i++) {
    H[i] = outs[i].H;
    W[i] = outs[i].W;
    data[i] = outs[i].data;
    ptrs[i] = outs[i].data;
  }
  int rc = check_images(n, H.data(), W.data(), data.data(), patch);
  if (rc) return rc;
  Batch b;
  rc = plan_batch(x->d, n, ptrs.data(), H.data(), W.data(), patch, layout, schedule, b);
  if (rc) return rc;
  if (decode_smem_bytes(x->d, (int)b.units.size()) > 227 * 1024)
    return fail(NLC_ERR_UNSUPPORTED, "too many coding units in one call (%zu)", b.units.size());
  const bool ring = x->d.shear && schedule == NLC_SCHED_WAVEFRONT;
  if (ring && b.ring_rows >= (1LL << 31) / kRingRowBytes)
    return fail(NLC_ERR_UNSUPPORTED, "batch too large for the sheared decoder's rings");
  nlc_plan* p = new nlc_plan();
  p->x = x;
  p->n = n;
  p->patch = patch;
  p->layout = layout;
  p->sched = schedule == NLC_SCHED_WAVEFRONT ? SCHED_WAVEFRONT : SCHED_RASTER;
  p->T = b.T;
  p->max_front = b.max_front;
  p->n_units = (int)b.units.size();
  p->px_per_cta = x->px_per_cta;
  const size_t need = layout_bufs(b, nullptr, p->cb, x->d_status, false, ring);
  cudaError_t e = cudaMalloc((void**)&p->d_buf, std::max<size_t>(need, 256));
  if (e != cudaSuccess) {
    delete p;
    return fail(NLC_ERR_CUDA, "cudaMalloc failed: %s", cudaGetErrorString(e));
  }
  layout_bufs(b, p->d_buf, p->cb, x->d_status, false, ring);
  if (!b.units.empty())
    e = cudaMemcpy((void*)p->cb.units, b.units.data(), b.units.size() * sizeof(Unit),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !b.images.empty())
    e = cudaMemcpy((void*)p->cb.images, b.images.data(), b.images.size() * sizeof(ImageRec),
                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(p->d_buf);
    delete p;
    return fail(NLC_ERR_CUDA, "unit table upload failed: %s", cudaGetErrorString(e));
  }
  // sets the decoder's shared-memory attribute for this batch, so runs need not
  p->gmax = decode_max_grid(model_view(x), p->n_units, x->sm_count, false, ring);
  if (p->gmax < 1) {
    cudaFree(p->d_buf);
    delete p;
    return fail(NLC_ERR_UNSUPPORTED, "decoder does not fit on an SM");
  }
  if (x->max_ctas > 0) p->gmax = std::min(p->gmax, x->max_ctas);
  p->grid = plan_grid(p, p->px_per_cta);
  *out = p;
  return NLC_OK;
}

extern "C" int nlc_plan_run(nlc_plan* p, const uint8_t* d_in, const uint64_t* d_offsets,
                            nlc_stream stream) {
  if (!p || (p->n > 0 && (!d_in || !d_offsets))) return fail(NLC_ERR_ARG, "bad arguments");
  if (reinterpret_cast<uintptr_t>(d_in) % 16) return fail(NLC_ERR_ARG, "d_in must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_packed(p->x, s);
  if (rc) return rc;
  p->cb.prof = prof_ptr(p->x);  // as of this call (a captured graph keeps it)
  p->cb.times = p->x->d_times;
  p->cb.n_times = p->x->n_times;
  p->cb.spin_limit = p->x->spin_limit;
  p->cb.mma_limit = p->x->mma_limit;
  CUDA_TRY(launch_decode(model_view(p->x), p->cb, d_in,
                         reinterpret_cast<const unsigned long long*>(d_offsets), p->layout,
                         p->patch, p->sched, (int)p->T, p->grid, s, false));
  return NLC_OK;
}

extern "C" int nlc_plan_tune(nlc_plan* p, const uint8_t* d_in, const uint64_t* d_offsets,
                             int reps, nlc_stream stream, int* h_px_per_cta, float* h_ms) {
  if (!p || reps < 1) return fail(NLC_ERR_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  static const int cand[] = {1, 2, 4, 8, 16, 32, 64, 128};
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  float best = 0.f;
  int best_ppc = p->px_per_cta, best_grid = p->grid, last_grid = -1, rc = NLC_OK;
  for (int c : cand) {
    const int grid = plan_grid(p, c);
    if (grid == last_grid) continue;  // same launch as the previous candidate
    last_grid = grid;
    p->grid = grid;
    if ((rc = nlc_plan_run(p, d_in, d_offsets, stream))) break;  // warm-up
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && rc == NLC_OK; r++) rc = nlc_plan_run(p, d_in, d_offsets, stream);
    cudaEventRecord(e1, s);
    if (rc) break;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      rc = fail(NLC_ERR_CUDA, "tuning run failed: %s", cudaGetErrorString(e));
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= (float)reps;
    if (best == 0.f || ms < best) {
      best = ms;
      best_ppc = c;
      best_grid = grid;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p->grid = best_grid;
  p->px_per_cta = best_ppc;
  if (rc) return rc;
  if (h_px_per_cta) *h_px_per_cta = best_ppc;
  if (h_ms) *h_ms = best;
  return NLC_OK;
}

extern "C" int nlc_plan_destroy(nlc_plan* p) {
  if (!p) return NLC_OK;
  cudaDeviceSynchronize();
  cudaFree(p->d_buf);
  delete p;
  return NLC_OK;
}
