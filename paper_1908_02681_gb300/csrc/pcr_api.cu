// libpcr host side: the C ABI declared in include/pcr.h (argument checks, per-view constants,
// framebuffer ownership, launches).
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pcr.h"
#include "pcr_batch.cuh"
#include "pcr_certified.cuh"
#include "pcr_kernels.cuh"
#include "pcr_project.cuh"

struct pcr_framebuffer {
  int32_t width, height;
  uint32_t flags;
  int device;
  unsigned long long* keys;  // width * height
  ulonglong2* accum;         // width * height (HQ only)
  ulonglong2* bounds;        // width * height (HQ only, allocated by the first pass 2 with band_bounds): pass 2's
                             // per-pixel accept bounds (pcr::k_band_bounds)
  uint32_t* status;          // device status word
  pcr::Tuning tuning;        // launch tuning of the point passes
  // device copy of the depth table of the view last rendered with the certified transform (loaded by the
  // passes with coalesced reads), re-uploaded when the view changes
  long long* d_table;
  pcr::DevView table_view;
  bool table_valid;
  // frames from host memory (pcr_render_frame_host): events, created by its first call (the copies go to the
  // device's upload queue, upload_stream)
  cudaEvent_t copy_events[9];  // [0]: start of the frame on the caller's stream; [1..8]: chunk k landed
  // band mask (pass 1 -> pass 2, see pcr::BandMask): two words per 64 points, grown on demand; valid for the
  // points, count, view and eps of the pass 1 that wrote it, until the framebuffer is cleared
  uint32_t* band_mask;
  uint64_t band_words;
  bool band_valid;
  const void* band_pts;
  uint64_t band_n;
  pcr::DevView band_view;
  uint32_t band_num, band_den;
};

namespace {

thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};

pcr_status fail(pcr_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

pcr_status cuda_fail(cudaError_t e, const char* what) {
  return fail(PCR_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// Streaming multiprocessor count of a device (cached per device id).
int sm_count(int device) {
  static std::mutex mu;
  static int cache[64] = {0};
  std::lock_guard<std::mutex> lock(mu);
  if (device < 0 || device >= 64) return 1;
  if (cache[device] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0) v = 1;
    cache[device] = v;
  }
  return cache[device];
}

// Blocks for a grid-stride kernel: enough to fill every SM `per_sm` times, no more than the work needs.
unsigned grid_for(uint64_t work_items, int threads, int device, int per_sm) {
  const uint64_t need = (work_items + threads - 1) / threads;
  const uint64_t cap = (uint64_t)sm_count(device) * per_sm;
  const uint64_t g = need < cap ? need : cap;
  return (unsigned)(g > 0 ? g : 1);
}

bool finite(double x) { return std::isfinite(x); }

// Validates a view and fills the device constants. Error text goes to the thread's last error.
pcr_status make_dev_view(const pcr_view* view, int32_t width, int32_t height, pcr::DevView* dv) {
  if (!view) return fail(PCR_ERR_INVALID_ARG, "view is NULL");
  for (int i = 0; i < 16; ++i)
    if (!finite(view->view_proj[i])) return fail(PCR_ERR_INVALID_ARG, "view_proj[%d] is not finite", i);
  const double near_ = view->near_plane, far_ = view->far_plane;
  if (!(near_ > 0.0) || !(far_ > near_) || !finite(far_))
    return fail(PCR_ERR_INVALID_ARG, "need 0 < near < far < inf (near=%g far=%g)", near_, far_);
  if (view->transform < PCR_TRANSFORM_EXACT || view->transform > PCR_TRANSFORM_DOUBLE_FLOAT)
    return fail(PCR_ERR_INVALID_ARG, "unknown transform %d", view->transform);
  if (view->reserved != 0) return fail(PCR_ERR_INVALID_ARG, "reserved field must be 0");
  std::memset(dv, 0, sizeof(*dv));
  const int rows[3] = {0, 1, 3};
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 4; ++c) dv->m[4 * r + c] = view->view_proj[4 * rows[r] + c];
  dv->near_ = near_;
  dv->far_ = far_;
  dv->depth_mode = view->depth_mode;
  dv->width = width;
  dv->height = height;
  dv->fwidth = (float)width;
  dv->fheight = (float)height;
  switch (view->depth_mode) {
    case PCR_DEPTH_LINEAR:
      dv->scale = 1099511627776.0 / (far_ - near_);  // 2^40 / (far - near), FP64
      dv->nq = (unsigned long long)std::floor(near_ * dv->scale);
      break;
    case PCR_DEPTH_METRIC:
      if (!(view->metric_scale > 0.0) || !finite(view->metric_scale))
        return fail(PCR_ERR_INVALID_ARG, "metric_scale must be positive and finite");
      dv->scale = view->metric_scale;
      dv->nq = 0;
      break;
    case PCR_DEPTH_PIECEWISE: {
      if (view->n_ranges < 1 || view->n_ranges > PCR_MAX_DEPTH_RANGES)
        return fail(PCR_ERR_INVALID_ARG, "n_ranges must be in 1..%d", PCR_MAX_DEPTH_RANGES);
      double base = 0.0;
      for (int k = 0; k < view->n_ranges; ++k) {
        const double lo = view->ranges[k][0], hi = view->ranges[k][1], res = view->ranges[k][2];
        if (!(lo >= 0.0) || !(hi > lo) || !finite(hi) || !(res > 0.0) || !finite(res))
          return fail(PCR_ERR_INVALID_ARG, "range %d invalid (need 0 <= lo < hi, res > 0)", k);
        if (k > 0 && lo < view->ranges[k - 1][1]) return fail(PCR_ERR_INVALID_ARG, "ranges overlap at %d", k);
        dv->lo[k] = lo;
        dv->hi[k] = hi;
        dv->res[k] = res;
        dv->base[k] = base;
        base += std::ceil((hi - lo) * res);
      }
      if (!(base < 9007199254740992.0)) return fail(PCR_ERR_INVALID_ARG, "piecewise ranges exceed 2^53 codes");
      dv->n_ranges = view->n_ranges;
      break;
    }
    default:
      return fail(PCR_ERR_INVALID_ARG, "unknown depth_mode %d", view->depth_mode);
  }
  return PCR_OK;
}

pcr_status check_fb(const pcr_framebuffer* fb) {
  if (!fb) return fail(PCR_ERR_INVALID_ARG, "framebuffer is NULL");
  return PCR_OK;
}

pcr_status check_points(const pcr_point* d_points, uint64_t n) {
  if (n == 0) return PCR_OK;
  if (!d_points) return fail(PCR_ERR_INVALID_ARG, "d_points is NULL");
  if (reinterpret_cast<uintptr_t>(d_points) & 15u) return fail(PCR_ERR_INVALID_ARG, "d_points is not 16-byte aligned");
  if (n >= (1ull << 40)) return fail(PCR_ERR_INVALID_ARG, "n must be below 2^40");
  return PCR_OK;
}

pcr_status after_launch(const char* what, uint64_t launches = 1) {
  g_launches.fetch_add(launches, std::memory_order_relaxed);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PCR_OK : cuda_fail(e, what);
}

// The device copy of the view's depth tables for the certified passes on fb (uploaded on `s` when the view
// differs from the last one; one table, or one per PIECEWISE range), or null (double-float transform, FP64
// kernels, or the upload failed: LINEAR and METRIC passes then read the table from their parameter block,
// PIECEWISE views run on the FP64 kernels).
const long long* fb_table(pcr_framebuffer* fb, const pcr::DevView& dv, int transform, cudaStream_t s) {
  if (transform != PCR_TRANSFORM_EXACT) return nullptr;
  const pcr::CertParams* P = nullptr;
  const long long* tables = nullptr;
  if (!pcr::cached_cert(dv, false, &P, &tables)) return nullptr;
  if (!fb->table_valid || std::memcmp(&fb->table_view, &dv, sizeof(dv)) != 0) {
    fb->table_valid = false;
    if (cudaMemcpyAsync(fb->d_table, tables, pcr::table_blocks(*P) * sizeof(P->F), cudaMemcpyHostToDevice, s) !=
        cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    fb->table_view = dv;
    fb->table_valid = true;
  }
  return fb->d_table;
}

// A band mask request for pass 1: on, its eps, and where the launch's first tile sits in the mask (a pass 1
// over a tile-aligned part of the frame's points).
struct BandRequest {
  bool on = false;
  uint32_t num = 1, den = 100;
  uint64_t tile_offset = 0;
};

// Makes the framebuffer's band mask hold `n_total` points (grown with cudaMalloc outside stream capture only);
// false when it cannot (then pass 1 writes no mask). The mask stops describing any points.
bool band_reserve(pcr_framebuffer* fb, uint64_t n_total, cudaStream_t s) {
  fb->band_valid = false;
  const uint64_t words = 2 * ((n_total + pcr::kTile - 1) / pcr::kTile);
  if (words <= fb->band_words) return true;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return false;
  }
  uint32_t* m = nullptr;
  if (cudaMalloc(&m, words * sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (fb->band_mask) {
    cudaStreamSynchronize(s);  // the old mask may still be read by pass 2 on this stream
    cudaFree(fb->band_mask);
  }
  fb->band_mask = m;
  fb->band_words = words;
  return true;
}

// Whether pass 1 of this view can write a band mask: the exact transform on a LINEAR or METRIC view of an HQ
// framebuffer.
bool band_applies(pcr_framebuffer* fb, const pcr::DevView& dv, int transform) {
  if (!(fb->flags & PCR_FB_HQ) || transform != PCR_TRANSFORM_EXACT) return false;
  const pcr::CertParams* P = nullptr;
  return pcr::cached_cert(dv, false, &P) && P->n_pw == 0;
}

// Launches pass 1 (atomic minimum) for a validated view. band.on: also write the band mask (the caller reserved
// it and records what it describes).
pcr_status launch_raster(pcr_framebuffer* fb, const pcr_point* d_points, uint64_t n, const pcr::DevView& dv,
                         int transform, cudaStream_t s, unsigned long long* stats = nullptr,
                         const BandRequest& band = BandRequest()) {
  const uint4* pts = reinterpret_cast<const uint4*>(d_points);
  if (transform == PCR_TRANSFORM_FP64) {
    pcr::k_raster_fp64<<<grid_for(n, 256, fb->device, 8), 256, 0, s>>>(pts, n, dv, fb->keys);
    return after_launch("k_raster_fp64");
  }
  const long long* table = fb_table(fb, dv, transform, s);
  const pcr::BandMask bm = pcr::band_mask(band.on ? fb->band_mask + 2 * band.tile_offset : nullptr, band.num,
                                          band.den, dv.nq);
  return pcr::launch_raster_certified(pts, n, dv, transform == PCR_TRANSFORM_DOUBLE_FLOAT, fb->keys, fb->status,
                                      sm_count(fb->device), s, stats, fb->tuning, table, bm)
             ? after_launch("k_raster_certified")
             : fail(PCR_ERR_CUDA, "certified raster launch failed");
}

// Pass 1 of n points with a band mask for eps num / den when it applies; records what the mask describes.
pcr_status launch_raster_band(pcr_framebuffer* fb, const pcr_point* d_points, uint64_t n, const pcr::DevView& dv,
                              int transform, uint32_t num, uint32_t den, cudaStream_t s) {
  BandRequest band;
  band.on = band_applies(fb, dv, transform) && band_reserve(fb, n, s);
  band.num = num;
  band.den = den;
  if (pcr_status st = launch_raster(fb, d_points, n, dv, transform, s, nullptr, band)) return st;
  if (band.on) {
    fb->band_valid = true;
    fb->band_pts = d_points;
    fb->band_n = n;
    fb->band_view = dv;
    fb->band_num = num;
    fb->band_den = den;
  }
  return PCR_OK;
}

// The framebuffer's per-pixel band bounds, allocated by the first call (outside stream capture only); null when
// they cannot be (pass 2 then tests against the stored keys).
ulonglong2* bounds_buffer(pcr_framebuffer* fb, cudaStream_t s) {
  if (fb->bounds) return fb->bounds;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return nullptr;
  }
  if (cudaMalloc(&fb->bounds, (uint64_t)fb->width * fb->height * sizeof(ulonglong2)) != cudaSuccess) {
    cudaGetLastError();
    fb->bounds = nullptr;
  }
  return fb->bounds;
}

pcr_status launch_hq(pcr_framebuffer* fb, const pcr_point* d_points, uint64_t n, const pcr::DevView& dv,
                     int transform, uint32_t eps_num, uint32_t eps_den, cudaStream_t s) {
  const uint4* pts = reinterpret_cast<const uint4*>(d_points);
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(fb->accum);
  if (transform == PCR_TRANSFORM_FP64) {
    pcr::k_hq_fp64<<<grid_for(n, 256, fb->device, 8), 256, 0, s>>>(pts, n, dv, fb->keys, acc, eps_num, eps_den);
    return after_launch("k_hq_fp64");
  }
  const long long* table = fb_table(fb, dv, transform, s);
  // pass 1's band mask, when it describes these points and view and an eps at least this one
  const bool band = fb->band_valid && transform == PCR_TRANSFORM_EXACT && fb->band_pts == d_points &&
                    fb->band_n == n && std::memcmp(&fb->band_view, &dv, sizeof(dv)) == 0 &&
                    (unsigned long long)eps_num * fb->band_den <= (unsigned long long)fb->band_num * eps_den;
  const int launched = pcr::launch_hq_certified(pts, n, dv, transform == PCR_TRANSFORM_DOUBLE_FLOAT, fb->keys, acc,
                                                eps_num, eps_den, fb->status, sm_count(fb->device), s, fb->tuning,
                                                table, band ? fb->band_mask : nullptr,
                                                fb->tuning.band_bounds ? bounds_buffer(fb, s) : nullptr);
  return after_launch("k_hq_certified", (uint64_t)launched);
}

}  // namespace

extern "C" {

pcr_status pcr_create_framebuffer(int32_t width, int32_t height, uint32_t flags, pcr_framebuffer** out) {
  if (!out) return fail(PCR_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (width < 1 || width > 16384 || height < 1 || height > 16384)
    return fail(PCR_ERR_INVALID_ARG, "width and height must be in 1..16384 (got %d x %d)", width, height);
  if (flags & ~PCR_FB_HQ) return fail(PCR_ERR_INVALID_ARG, "unknown flags 0x%x", flags);
  pcr_framebuffer* fb = new (std::nothrow) pcr_framebuffer();
  if (!fb) return fail(PCR_ERR_OOM, "host allocation failed");
  fb->width = width;
  fb->height = height;
  fb->flags = flags;
  cudaError_t e = cudaGetDevice(&fb->device);
  if (e != cudaSuccess) {
    delete fb;
    return cuda_fail(e, "cudaGetDevice");
  }
  const uint64_t npx = (uint64_t)width * (uint64_t)height;
  e = cudaMalloc(&fb->keys, npx * sizeof(unsigned long long));
  if (e == cudaSuccess && (flags & PCR_FB_HQ)) e = cudaMalloc(&fb->accum, npx * sizeof(ulonglong2));
  if (e == cudaSuccess) e = cudaMalloc(&fb->status, 256);
  if (e == cudaSuccess) e = cudaMalloc(&fb->d_table, pcr::kMaxRanges * sizeof(pcr::CertParams::F));
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(fb->keys);
    cudaFree(fb->accum);
    cudaFree(fb->bounds);
    cudaFree(fb->status);
    cudaFree(fb->d_table);
    delete fb;
    return e == cudaErrorMemoryAllocation ? fail(PCR_ERR_OOM, "cudaMalloc of %llu pixels failed", (unsigned long long)npx)
                                          : cuda_fail(e, "cudaMalloc");
  }
  e = cudaMemset(fb->status, 0, 256);
  if (e == cudaSuccess) {
    pcr::k_clear<<<grid_for(npx / 2 + 1, 256, fb->device, 4), 256>>>(fb->keys, fb->accum, npx);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    e = cudaGetLastError();
  }
  // wait for the clear on the stream it ran on (not the whole device: other streams keep running)
  if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
  if (e != cudaSuccess) {
    pcr_destroy_framebuffer(fb);
    return cuda_fail(e, "framebuffer clear");
  }
  *out = fb;
  return PCR_OK;
}

pcr_status pcr_destroy_framebuffer(pcr_framebuffer* fb) {
  if (!fb) return PCR_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(fb->device);
  cudaDeviceSynchronize();
  cudaFree(fb->keys);
  cudaFree(fb->accum);
  cudaFree(fb->bounds);
  cudaFree(fb->status);
  cudaFree(fb->d_table);
  cudaFree(fb->band_mask);
  for (cudaEvent_t e : fb->copy_events)
    if (e) cudaEventDestroy(e);
  cudaSetDevice(prev);
  delete fb;
  return PCR_OK;
}

pcr_status pcr_set_tuning(pcr_framebuffer* fb, const pcr_tuning* tuning) {
  if (pcr_status st = check_fb(fb)) return st;
  if (!tuning) {
    fb->tuning = pcr::Tuning();
    return PCR_OK;
  }
  if (tuning->merge_same_pixel != 0 && tuning->merge_same_pixel != 1)
    return fail(PCR_ERR_INVALID_ARG, "merge_same_pixel must be 0 or 1");
  if (tuning->blocks_per_sm < 1 || tuning->blocks_per_sm > 32) return fail(PCR_ERR_INVALID_ARG, "blocks_per_sm must be in 1..32");
  if (tuning->staging != 0 && tuning->staging != 1) return fail(PCR_ERR_INVALID_ARG, "staging must be 0 or 1");
  if (tuning->band_filter != 0 && tuning->band_filter != 1) return fail(PCR_ERR_INVALID_ARG, "band_filter must be 0 or 1");
  if (tuning->band_eps_den == 0 || tuning->band_eps_den > (1u << 20))
    return fail(PCR_ERR_INVALID_ARG, "band_eps_den must be in 1..2^20");
  fb->tuning.merge = tuning->merge_same_pixel;
  fb->tuning.blocks_per_sm = tuning->blocks_per_sm;
  fb->tuning.staging = tuning->staging;
  if (tuning->band_bounds != 0 && tuning->band_bounds != 1) return fail(PCR_ERR_INVALID_ARG, "band_bounds must be 0 or 1");
  fb->tuning.band_filter = tuning->band_filter;
  fb->tuning.band_bounds = tuning->band_bounds;
  fb->tuning.band_num = tuning->band_eps_num;
  fb->tuning.band_den = tuning->band_eps_den;
  return PCR_OK;
}

pcr_status pcr_get_tuning(const pcr_framebuffer* fb, pcr_tuning* tuning) {
  if (pcr_status st = check_fb(fb)) return st;
  if (!tuning) return fail(PCR_ERR_INVALID_ARG, "tuning is NULL");
  tuning->merge_same_pixel = fb->tuning.merge;
  tuning->blocks_per_sm = fb->tuning.blocks_per_sm;
  tuning->staging = fb->tuning.staging;
  tuning->band_filter = fb->tuning.band_filter;
  tuning->band_bounds = fb->tuning.band_bounds;
  tuning->band_eps_num = fb->tuning.band_num;
  tuning->band_eps_den = fb->tuning.band_den;
  return PCR_OK;
}

pcr_status pcr_autotune(pcr_framebuffer* fb, const pcr_point* d_points, uint64_t n, const pcr_view* view,
                        pcr_stream_t stream, pcr_tuning* best) {
  if (pcr_status st = check_fb(fb)) return st;
  if (pcr_status st = check_points(d_points, n)) return st;
  if (n == 0) return fail(PCR_ERR_INVALID_ARG, "autotuning needs points");
  pcr::DevView dv;
  if (pcr_status st = make_dev_view(view, fb->width, fb->height, &dv)) return st;
  const bool hq = (fb->flags & PCR_FB_HQ) && dv.depth_mode != PCR_DEPTH_PIECEWISE;
  const cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return fail(PCR_ERR_CUDA, "cudaEventCreate failed");
  }
  const pcr::Tuning saved = fb->tuning;
  pcr::Tuning best_t = saved;
  float best_ms = 3.0e38f;
  pcr_status st = PCR_OK;
  for (int cand = 0; cand < (hq ? 64 : 16) && st == PCR_OK; ++cand) {
    fb->tuning.merge = cand & 1;
    fb->tuning.staging = (cand >> 1) & 1;
    fb->tuning.blocks_per_sm = 2 + 2 * ((cand >> 2) & 3);  // 2, 4, 6, 8
    fb->tuning.band_filter = (cand >> 4) & 1;               // HQ: band records (eps 1 / 100) on and off
    fb->tuning.band_bounds = cand >> 5;                     // HQ: pass 2's per-pixel bounds on and off
    fb->tuning.band_num = 1;
    fb->tuning.band_den = 100;
    float run_best = 3.0e38f;
    for (int rep = 0; rep < 2 && st == PCR_OK; ++rep) {
      if ((st = pcr_clear(fb, stream)) != PCR_OK) break;
      cudaEventRecord(e0, s);
      st = hq && fb->tuning.band_filter ? launch_raster_band(fb, d_points, n, dv, view->transform, 1, 100, s)
                                        : launch_raster(fb, d_points, n, dv, view->transform, s);
      if (st == PCR_OK && hq) st = launch_hq(fb, d_points, n, dv, view->transform, 1, 100, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "autotune timing");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      run_best = ms < run_best ? ms : run_best;
    }
    if (st != PCR_OK) break;
    if (run_best < best_ms) {
      best_ms = run_best;
      best_t = fb->tuning;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  fb->tuning = st == PCR_OK ? best_t : saved;
  if (st == PCR_OK) st = pcr_clear(fb, stream);
  if (st == PCR_OK) {
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "autotune");
  }
  if (st == PCR_OK && best) {
    best->merge_same_pixel = fb->tuning.merge;
    best->blocks_per_sm = fb->tuning.blocks_per_sm;
    best->staging = fb->tuning.staging;
    best->band_filter = fb->tuning.band_filter;
    best->band_bounds = fb->tuning.band_bounds;
    best->band_eps_num = fb->tuning.band_num;
    best->band_eps_den = fb->tuning.band_den;
  }
  return st;
}

pcr_status pcr_framebuffer_info(const pcr_framebuffer* fb, int32_t* width, int32_t* height, uint32_t* flags) {
  if (pcr_status st = check_fb(fb)) return st;
  if (width) *width = fb->width;
  if (height) *height = fb->height;
  if (flags) *flags = fb->flags;
  return PCR_OK;
}

pcr_status pcr_clear(pcr_framebuffer* fb, pcr_stream_t stream) {
  if (pcr_status st = check_fb(fb)) return st;
  fb->band_valid = false;
  const uint64_t npx = (uint64_t)fb->width * fb->height;
  pcr::k_clear<<<grid_for(npx / 2 + 1, 256, fb->device, 4), 256, 0, (cudaStream_t)stream>>>(fb->keys, fb->accum, npx);
  return after_launch("k_clear");
}

pcr_status pcr_render_atomicmin(pcr_framebuffer* fb, const pcr_point* d_points, uint64_t n, const pcr_view* view,
                                pcr_stream_t stream) {
  if (pcr_status st = check_fb(fb)) return st;
  if (pcr_status st = check_points(d_points, n)) return st;
  pcr::DevView dv;
  if (pcr_status st = make_dev_view(view, fb->width, fb->height, &dv)) return st;
  if (n == 0) return PCR_OK;
  if (fb->tuning.band_filter)
    return launch_raster_band(fb, d_points, n, dv, view->transform, fb->tuning.band_num, fb->tuning.band_den,
                              (cudaStream_t)stream);
  return launch_raster(fb, d_points, n, dv, view->transform, (cudaStream_t)stream);
}

pcr_status pcr_project_points(const pcr_point* d_points, uint64_t n, const pcr_view* view, int32_t width,
                              int32_t height, uint32_t* d_pixel, uint64_t* d_key, pcr_stream_t stream) {
  if (pcr_status st = check_points(d_points, n)) return st;
  if (width < 1 || width > 16384 || height < 1 || height > 16384)
    return fail(PCR_ERR_INVALID_ARG, "width and height must be in 1..16384 (got %d x %d)", width, height);
  if (n > 0 && (!d_pixel || !d_key)) return fail(PCR_ERR_INVALID_ARG, "d_pixel and d_key must not be NULL");
  pcr::DevView dv;
  if (pcr_status st = make_dev_view(view, width, height, &dv)) return st;
  if (n == 0) return PCR_OK;
  int device = 0;
  if (const cudaError_t e = cudaGetDevice(&device)) return cuda_fail(e, "cudaGetDevice");
  const cudaStream_t s = (cudaStream_t)stream;
  const uint4* pts = reinterpret_cast<const uint4*>(d_points);
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(d_key);
  const unsigned grid = grid_for(n, 256, device, 8);
  const pcr::CertParams* P = nullptr;
  const long long* tables = nullptr;
  const bool approx = view->transform == PCR_TRANSFORM_DOUBLE_FLOAT;
  if (view->transform == PCR_TRANSFORM_FP64 || !pcr::cached_cert(dv, approx, &P, &tables)) {
    pcr::k_project_fp64<<<grid, 256, 0, s>>>(pts, n, dv, d_pixel, keys);
  } else if (P->n_pw > 0) {
    // PIECEWISE: the ranges' tables in a stream-ordered temporary device copy
    const size_t bytes = (size_t)P->n_pw * sizeof(P->F);
    void* d_tab = nullptr;
    cudaError_t e = cudaMallocAsync(&d_tab, bytes, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_tab, tables, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      auto kernel = P->n_pw > 2 ? pcr::k_project_cert<false, 2> : pcr::k_project_cert<false, 1>;
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e == cudaSuccess) kernel<<<grid, 256, bytes, s>>>(pts, n, *P, d_pixel, keys, (const long long*)d_tab);
      if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (d_tab) cudaFreeAsync(d_tab, s);
    if (e != cudaSuccess) return cuda_fail(e, "piecewise projection");
  } else if (approx)
    pcr::k_project_cert<true><<<grid, 256, 0, s>>>(pts, n, *P, d_pixel, keys);
  else
    pcr::k_project_cert<false><<<grid, 256, 0, s>>>(pts, n, *P, d_pixel, keys);
  return after_launch("k_project");
}

pcr_status pcr_render_atomicmin_stats(pcr_framebuffer* fb, const pcr_point* d_points, uint64_t n,
                                      const pcr_view* view, uint64_t* d_counts, pcr_stream_t stream) {
  if (pcr_status st = check_fb(fb)) return st;
  if (pcr_status st = check_points(d_points, n)) return st;
  if (!d_counts || (reinterpret_cast<uintptr_t>(d_counts) & 7u)) return fail(PCR_ERR_INVALID_ARG, "d_counts invalid");
  pcr::DevView dv;
  if (pcr_status st = make_dev_view(view, fb->width, fb->height, &dv)) return st;
  if (n == 0) return PCR_OK;
  return launch_raster(fb, d_points, n, dv, view->transform, (cudaStream_t)stream,
                       reinterpret_cast<unsigned long long*>(d_counts));
}

namespace {

// Checks shared by the two HQ entry points; fills dv.
pcr_status check_hq(pcr_framebuffer* fb, const pcr_point* d_points, uint64_t n, const pcr_view* view, uint32_t eps_num,
                    uint32_t eps_den, pcr::DevView* dv) {
  if (pcr_status st = check_fb(fb)) return st;
  if (!(fb->flags & PCR_FB_HQ)) return fail(PCR_ERR_INVALID_ARG, "framebuffer was created without PCR_FB_HQ");
  if (pcr_status st = check_points(d_points, n)) return st;
  if (pcr_status st = make_dev_view(view, fb->width, fb->height, dv)) return st;
  if (dv->depth_mode == PCR_DEPTH_PIECEWISE)
    return fail(PCR_ERR_INVALID_ARG, "HQ splatting needs codes proportional to depth (LINEAR or METRIC)");
  if (eps_den == 0 || eps_den > (1u << 20)) return fail(PCR_ERR_INVALID_ARG, "eps_den must be in 1..2^20");
  // eps_num * (qmin + Nq) must not wrap for any qmin < 2^40
  const long double lim = (long double)eps_num * ((long double)(1ull << 40) + (long double)dv->nq);
  if (lim >= 18446744073709551616.0L) return fail(PCR_ERR_INVALID_ARG, "eps_num * (2^40 + Nq) must be below 2^64");
  return PCR_OK;
}

}  // namespace

pcr_status pcr_render_hq_splat(pcr_framebuffer* fb, const pcr_point* d_points, uint64_t n, const pcr_view* view,
                               uint32_t eps_num, uint32_t eps_den, pcr_stream_t stream) {
  pcr::DevView dv;
  if (pcr_status st = check_hq(fb, d_points, n, view, eps_num, eps_den, &dv)) return st;
  if (n == 0) return PCR_OK;
  const cudaStream_t s = (cudaStream_t)stream;
  const pcr_status st = fb->tuning.band_filter ? launch_raster_band(fb, d_points, n, dv, view->transform, eps_num,
                                                                    eps_den, s)
                                               : launch_raster(fb, d_points, n, dv, view->transform, s);
  if (st != PCR_OK) return st;
  return launch_hq(fb, d_points, n, dv, view->transform, eps_num, eps_den, s);
}

pcr_status pcr_hq_accumulate(pcr_framebuffer* fb, const pcr_point* d_points, uint64_t n, const pcr_view* view,
                             uint32_t eps_num, uint32_t eps_den, pcr_stream_t stream) {
  pcr::DevView dv;
  if (pcr_status st = check_hq(fb, d_points, n, view, eps_num, eps_den, &dv)) return st;
  if (n == 0) return PCR_OK;
  return launch_hq(fb, d_points, n, dv, view->transform, eps_num, eps_den, (cudaStream_t)stream);
}

pcr_status pcr_resolve(pcr_framebuffer* fb, uint32_t* d_rgba_out, uint32_t background_rgba, int32_t clear_after,
                       pcr_stream_t stream) {
  if (pcr_status st = check_fb(fb)) return st;
  if (!d_rgba_out) return fail(PCR_ERR_INVALID_ARG, "d_rgba_out is NULL");
  if (!(fb->flags & PCR_FB_HQ)) return pcr_resolve_basic(fb, d_rgba_out, background_rgba, clear_after, stream);
  const uint64_t npx = (uint64_t)fb->width * fb->height;
  if (clear_after) fb->band_valid = false;
  pcr::k_resolve_hq<<<grid_for(npx, 256, fb->device, 4), 256, 0, (cudaStream_t)stream>>>(
      fb->accum, fb->keys, d_rgba_out, npx, background_rgba, clear_after != 0, fb->status);
  return after_launch("k_resolve_hq");
}

pcr_status pcr_resolve_basic(pcr_framebuffer* fb, uint32_t* d_rgba_out, uint32_t background_rgba,
                             int32_t clear_after, pcr_stream_t stream) {
  if (pcr_status st = check_fb(fb)) return st;
  if (!d_rgba_out) return fail(PCR_ERR_INVALID_ARG, "d_rgba_out is NULL");
  const uint64_t npx = (uint64_t)fb->width * fb->height;
  if (clear_after) fb->band_valid = false;
  pcr::k_resolve_basic<<<grid_for(npx, 256, fb->device, 4), 256, 0, (cudaStream_t)stream>>>(
      fb->keys, fb->accum, d_rgba_out, npx, background_rgba, clear_after != 0);
  return after_launch("k_resolve_basic");
}

pcr_status pcr_resolve_both(pcr_framebuffer* fb, uint32_t* d_rgba_basic, uint32_t* d_rgba_hq, uint32_t background_rgba,
                            int32_t clear_after, pcr_stream_t stream) {
  if (pcr_status st = check_fb(fb)) return st;
  if (!(fb->flags & PCR_FB_HQ)) return fail(PCR_ERR_INVALID_ARG, "framebuffer was created without PCR_FB_HQ");
  if (!d_rgba_basic || !d_rgba_hq) return fail(PCR_ERR_INVALID_ARG, "an output image is NULL");
  const uint64_t npx = (uint64_t)fb->width * fb->height;
  if (clear_after) fb->band_valid = false;
  pcr::k_resolve_both<<<grid_for(npx, 256, fb->device, 4), 256, 0, (cudaStream_t)stream>>>(
      fb->keys, fb->accum, d_rgba_basic, d_rgba_hq, npx, background_rgba, clear_after != 0, fb->status);
  return after_launch("k_resolve_both");
}

pcr_status pcr_framebuffer_keys(const pcr_framebuffer* fb, const uint64_t** d_keys, const uint64_t** d_accum) {
  if (pcr_status st = check_fb(fb)) return st;
  if (d_keys) *d_keys = reinterpret_cast<const uint64_t*>(fb->keys);
  if (d_accum) *d_accum = reinterpret_cast<const uint64_t*>(fb->accum);
  return PCR_OK;
}

pcr_status pcr_get_device_status(pcr_framebuffer* fb, pcr_stream_t stream) {
  if (pcr_status st = check_fb(fb)) return st;
  const cudaStream_t s = (cudaStream_t)stream;
  uint32_t word = 0;
  cudaError_t e = cudaMemcpyAsync(&word, fb->status, sizeof(word), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemsetAsync(fb->status, 0, sizeof(word), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "reading the device status");
  if (word & pcr::kStatusOverflow)
    return fail(PCR_ERR_OVERFLOW, "an HQ pixel received more than 2^24 contributing fragments");
  if (word & pcr::kStatusTimeout) return fail(PCR_ERR_TIMEOUT, "a bounded device-side wait gave up");
  return PCR_OK;
}

namespace {

// The device's upload queue for frames from host memory: their copies share the host-to-device link, so they
// run back to back in call order, and each frame's passes overlap the next frame's upload. (With one copy
// stream per framebuffer, two frames in flight uploaded side by side, finished together, and left the link idle
// while both computed: 91-92 % of the link's rate end to end.) Created by the first frame on the device; lives
// as long as the process.
cudaStream_t upload_stream(int device, cudaError_t* err) {
  static std::mutex mu;
  static cudaStream_t streams[64] = {};
  std::lock_guard<std::mutex> lock(mu);
  *err = cudaSuccess;
  if (device < 0 || device >= 64) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  if (!streams[device]) *err = cudaStreamCreateWithFlags(&streams[device], cudaStreamNonBlocking);
  return streams[device];
}

}  // namespace

pcr_status pcr_render_frame_host(pcr_framebuffer* fb, const pcr_point* h_points, uint64_t n, const pcr_view* view,
                                 uint32_t eps_num, uint32_t eps_den, uint32_t background_rgba, pcr_point* d_points,
                                 uint32_t* d_images, uint32_t* h_basic, uint32_t* h_hq, pcr_stream_t stream) {
  const bool hq = fb && (fb->flags & PCR_FB_HQ);
  pcr::DevView dv;
  if (hq) {
    if (pcr_status st = check_hq(fb, d_points, n, view, eps_num, eps_den, &dv)) return st;
  } else {
    if (pcr_status st = check_fb(fb)) return st;
    if (pcr_status st = check_points(d_points, n)) return st;
    if (pcr_status st = make_dev_view(view, fb->width, fb->height, &dv)) return st;
  }
  if (n > 0 && !h_points) return fail(PCR_ERR_INVALID_ARG, "h_points is NULL");
  if (!d_images || !h_basic || (hq && !h_hq)) return fail(PCR_ERR_INVALID_ARG, "d_images and the host images are required");
  const cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  const cudaStream_t up = upload_stream(fb->device, &e);
  if (e != cudaSuccess) return cuda_fail(e, "upload stream");
  if (!fb->copy_events[8]) {  // first call on this framebuffer
    for (int k = 0; k < 9 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&fb->copy_events[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      for (cudaEvent_t& ev : fb->copy_events) {
        if (ev) cudaEventDestroy(ev);
        ev = nullptr;
      }
      return cuda_fail(e, "copy events");
    }
  }
  // the copies into d_points wait for earlier work on the caller's stream (which may still read them)
  e = cudaEventRecord(fb->copy_events[0], s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(up, fb->copy_events[0], 0);
  if (e != cudaSuccess) return cuda_fail(e, "frame start");
  // up to 8 chunks: pass 1 of chunk k runs while chunk k + 1 is still being copied. Chunk bounds are multiples
  // of 64 points, so that each chunk's band mask (HQ frames) is its part of the frame's mask.
  const uint64_t chunks = n < (8ull << 20) ? 1 : 8;
  BandRequest band;
  band.on = hq && n > 0 && fb->tuning.band_filter && band_applies(fb, dv, view->transform) && band_reserve(fb, n, s);
  band.num = eps_num;
  band.den = eps_den;
  auto bound = [&](uint64_t k) { return k >= chunks ? n : (n * k / chunks) / pcr::kTile * pcr::kTile; };
  for (uint64_t k = 0; k < chunks && n > 0; ++k) {
    const uint64_t lo = bound(k), hi = bound(k + 1);
    if (hi == lo) continue;
    e = cudaMemcpyAsync(d_points + lo, h_points + lo, (hi - lo) * sizeof(pcr_point), cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess) e = cudaEventRecord(fb->copy_events[1 + k], up);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, fb->copy_events[1 + k], 0);
    if (e != cudaSuccess) return cuda_fail(e, "point upload");
    band.tile_offset = lo / pcr::kTile;
    if (pcr_status st = launch_raster(fb, d_points + lo, hi - lo, dv, view->transform, s, nullptr, band)) return st;
  }
  if (band.on) {
    fb->band_valid = true;
    fb->band_pts = d_points;
    fb->band_n = n;
    fb->band_view = dv;
    fb->band_num = eps_num;
    fb->band_den = eps_den;
  }
  if (hq && n > 0)
    if (pcr_status st = launch_hq(fb, d_points, n, dv, view->transform, eps_num, eps_den, s)) return st;
  const uint64_t npx = (uint64_t)fb->width * fb->height;
  if (pcr_status st = hq ? pcr_resolve_both(fb, d_images, d_images + npx, background_rgba, 1, stream)
                         : pcr_resolve_basic(fb, d_images, background_rgba, 1, stream))
    return st;
  e = cudaMemcpyAsync(h_basic, d_images, npx * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && hq) e = cudaMemcpyAsync(h_hq, d_images + npx, npx * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "image download");
  return PCR_OK;
}

pcr_status pcr_check_bounded_wait(pcr_framebuffer* fb, uint32_t rounds, pcr_stream_t stream) {
  if (pcr_status st = check_fb(fb)) return st;
  if (rounds > pcr::kSpinLimit) return fail(PCR_ERR_INVALID_ARG, "rounds must be at most %u", pcr::kSpinLimit);
  pcr::k_wait_check<<<1, 32, 0, (cudaStream_t)stream>>>(fb->status, rounds ? rounds : pcr::kSpinLimit);
  return after_launch("k_wait_check");
}

const char* pcr_status_string(pcr_status status) {
  switch (status) {
    case PCR_OK: return "PCR_OK";
    case PCR_ERR_INVALID_ARG: return "PCR_ERR_INVALID_ARG: invalid argument";
    case PCR_ERR_CUDA: return "PCR_ERR_CUDA: CUDA runtime error";
    case PCR_ERR_OOM: return "PCR_ERR_OOM: device allocation failed";
    case PCR_ERR_OVERFLOW: return "PCR_ERR_OVERFLOW: HQ fragment count above 2^24 in a pixel";
    case PCR_ERR_TIMEOUT: return "PCR_ERR_TIMEOUT: bounded device wait expired";
  }
  return "unknown pcr_status";
}

const char* pcr_last_error_message(void) { return g_last_error.c_str(); }

uint64_t pcr_kernel_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"

#include "pcr_batch_api.inc"
#include "pcr_server.inc"
#include "pcr_noalloc.inc"
