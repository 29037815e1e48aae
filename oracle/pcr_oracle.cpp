// Oracle for the point-cloud rasterizer of Schuetz & Wimmer, "Rendering Point Clouds with Compute
// Shaders" (arXiv 1908.02681). TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU
// baseline leg of the benchmark may call it; the rendering library never does.
//
// Plain, single-threaded, FP64 C++ with no blocking, fusion or reordering: every function walks the
// points (or pixels) once in input order and applies the definition directly. It shares no code with
// the CUDA library. Build with -ffp-contract=off so that the only fused multiply-adds are the explicit
// std::fma / std::fmaf calls below.
//
// What it computes (paper Section 2.1 "Rasterization via AtomicMin", Section 2.2 "High-Quality
// Splatting"), with the readings taken where the paper is silent:
//   * project: clip = M (x, y, z, 1) with depth in double precision (Sections 1 and 2.1); clip x, y, w
//     each as fma(M[r][2], Z, fma(M[r][1], Y, fma(M[r][0], X, M[r][3]))).
//   * cull unless near <= w < far (NaN culled); pixel from the float-rounded clip values:
//     fx = fmaf(fcx / fw, 0.5, 0.5) * W, kept when 0 <= fx < W (same for y), px = (int)fx, row 0 = bottom.
//   * depth to a 40-bit integer (Section 2.1): linear mode t = (w - near) * s with s = 2^40 / (far - near);
//     metric mode t = w * metric_scale (the paper's "multiply by 1000, keep the integer part");
//     piecewise mode: per-range affine maps, see oracle_quantise_piecewise. q = min(floor(t), 2^40 - 2).
//   * key = (q << 24) | (rgba & 0xFFFFFF): depth in the most significant bits, colour in the least
//     significant 24 (Section 2.1), so equal depths resolve to the smaller colour value.
//   * framebuffer pixel = minimum key over the fragments that land on it; empty = 0xFFFFFFFFFFFFFFFF.
//   * resolve (Section 2.1, second compute shader): colour of the stored key, background where empty.
//   * high-quality splatting (Section 2.2): a fragment contributes when its linear depth is at most
//     eps (1 %) larger than the pixel's closest depth, tested exactly on integers as
//     eps_den * (q - qmin) <= eps_num * (qmin + Nq), Nq = floor(near * s) in linear mode, 0 in metric
//     mode; contributing fragments add R, G, B and 1 to per-pixel sums; the resolve divides
//     (round half up).
#include <cmath>
#include <cstdint>
#include <cstring>

namespace {

constexpr uint64_t kEmpty = 0xFFFFFFFFFFFFFFFFull;
constexpr uint64_t kQMax = (1ull << 40) - 2;  // largest depth code; keeps every key below kEmpty

struct OView {
  double M[16];  // row-major view-projection
  double near_, far_;
  int depth_mode;  // 0 linear, 1 metric, 2 piecewise
  double metric_scale;
  // piecewise mode: ranges [lo_k, hi_k) with resolution res_k (units per metre), consecutive offsets
  int n_ranges;
  double pw_lo[8], pw_hi[8], pw_res[8];
  int W, H;
};

struct Frag {
  bool visible;
  int64_t pixel;  // py * W + px
  uint64_t q;
  uint64_t key;
};

inline void read_point(const unsigned char* pts, uint64_t i, float* x, float* y, float* z, uint32_t* rgba) {
  std::memcpy(x, pts + i * 16 + 0, 4);
  std::memcpy(y, pts + i * 16 + 4, 4);
  std::memcpy(z, pts + i * 16 + 8, 4);
  std::memcpy(rgba, pts + i * 16 + 12, 4);
}

// Piecewise depth code of a depth d (Section 2.1: sub-ranges with different precision, e.g. [0, 10 m]
// in nanometres, [10 m, 10 km] in micrometres, [10 km, 10 000 km] in millimetres). Range k covers
// [lo_k, hi_k) at res_k codes per metre and starts where range k-1's codes end:
//   code = base_k + floor((d - lo_k) * res_k), base_0 = 0, base_k = base_{k-1} + ceil((hi_{k-1} - lo_{k-1}) * res_{k-1}).
// Depths outside every range are culled (returns false).
bool quantise_piecewise(const OView& v, double d, double* t) {
  double base = 0.0;
  for (int k = 0; k < v.n_ranges; ++k) {
    if (d >= v.pw_lo[k] && d < v.pw_hi[k]) {
      *t = base + std::floor((d - v.pw_lo[k]) * v.pw_res[k]);
      return true;
    }
    base += std::ceil((v.pw_hi[k] - v.pw_lo[k]) * v.pw_res[k]);
  }
  return false;
}

inline double linear_scale(const OView& v) { return 1099511627776.0 / (v.far_ - v.near_); }  // 2^40 / (far - near)

Frag project(const OView& v, float x, float y, float z, uint32_t rgba) {
  Frag f{false, -1, 0, 0};
  const double X = x, Y = y, Z = z;
  const double* M = v.M;
  const double cx = std::fma(M[2], Z, std::fma(M[1], Y, std::fma(M[0], X, M[3])));
  const double cy = std::fma(M[6], Z, std::fma(M[5], Y, std::fma(M[4], X, M[7])));
  const double w = std::fma(M[14], Z, std::fma(M[13], Y, std::fma(M[12], X, M[15])));
  if (!(w >= v.near_ && w < v.far_)) return f;
  const float fw = (float)w, fcx = (float)cx, fcy = (float)cy;
  const float fx = std::fmaf(fcx / fw, 0.5f, 0.5f) * (float)v.W;
  const float fy = std::fmaf(fcy / fw, 0.5f, 0.5f) * (float)v.H;
  if (!(fx >= 0.0f && fx < (float)v.W && fy >= 0.0f && fy < (float)v.H)) return f;
  const int px = (int)fx, py = (int)fy;
  double t;
  if (v.depth_mode == 0) {
    const double d = w - v.near_;
    t = d * linear_scale(v);
  } else if (v.depth_mode == 1) {
    t = w * v.metric_scale;
  } else {
    if (!quantise_piecewise(v, w, &t)) return f;
  }
  double ft = std::floor(t);
  uint64_t q = ft >= (double)kQMax ? kQMax : (uint64_t)ft;
  f.visible = true;
  f.pixel = (int64_t)py * v.W + px;
  f.q = q;
  f.key = (q << 24) | (uint64_t)(rgba & 0xFFFFFFu);
  return f;
}

bool make_view(const double* M, double near_, double far_, int depth_mode, double metric_scale, int n_ranges,
               const double* ranges, int W, int H, OView* v) {
  if (!M || W <= 0 || H <= 0) return false;
  if (!(near_ > 0.0) || !(far_ > near_) || !std::isfinite(far_)) return false;
  if (depth_mode < 0 || depth_mode > 2) return false;
  if (depth_mode == 1 && !(metric_scale > 0.0 && std::isfinite(metric_scale))) return false;
  for (int k = 0; k < 16; ++k)
    if (!std::isfinite(M[k])) return false;
  std::memcpy(v->M, M, sizeof(v->M));
  v->near_ = near_;
  v->far_ = far_;
  v->depth_mode = depth_mode;
  v->metric_scale = metric_scale;
  v->n_ranges = 0;
  if (depth_mode == 2) {
    if (n_ranges < 1 || n_ranges > 8 || !ranges) return false;
    v->n_ranges = n_ranges;
    for (int k = 0; k < n_ranges; ++k) {
      v->pw_lo[k] = ranges[3 * k];
      v->pw_hi[k] = ranges[3 * k + 1];
      v->pw_res[k] = ranges[3 * k + 2];
      if (!(v->pw_lo[k] >= 0.0 && v->pw_hi[k] > v->pw_lo[k] && std::isfinite(v->pw_hi[k]) && v->pw_res[k] > 0.0 &&
            std::isfinite(v->pw_res[k])))
        return false;
      if (k > 0 && v->pw_lo[k] < v->pw_hi[k - 1]) return false;
    }
  }
  v->W = W;
  v->H = H;
  return true;
}

}  // namespace

extern "C" {

// Per-point projection: pixel (-1 when culled), depth code q and key.
int oracle_project(const void* points, uint64_t n, const double* M, double near_, double far_, int depth_mode,
                   double metric_scale, int n_ranges, const double* ranges, int W, int H, int64_t* pixel,
                   uint64_t* q, uint64_t* key) {
  OView v;
  if (!make_view(M, near_, far_, depth_mode, metric_scale, n_ranges, ranges, W, H, &v)) return 1;
  const unsigned char* p = (const unsigned char*)points;
  for (uint64_t i = 0; i < n; ++i) {
    float x, y, z;
    uint32_t c;
    read_point(p, i, &x, &y, &z, &c);
    Frag f = project(v, x, y, z, c);
    pixel[i] = f.visible ? f.pixel : -1;
    q[i] = f.q;
    key[i] = f.visible ? f.key : kEmpty;
  }
  return 0;
}

// Basic rasterization (Section 2.1): fb[pixel] = min(fb[pixel], key) over the points in order.
// fb holds W*H keys and is NOT cleared here (oracle_clear does that), so several calls accumulate.
int oracle_render_atomicmin(const void* points, uint64_t n, const double* M, double near_, double far_,
                            int depth_mode, double metric_scale, int n_ranges, const double* ranges, int W, int H,
                            uint64_t* fb) {
  OView v;
  if (!make_view(M, near_, far_, depth_mode, metric_scale, n_ranges, ranges, W, H, &v)) return 1;
  const unsigned char* p = (const unsigned char*)points;
  for (uint64_t i = 0; i < n; ++i) {
    float x, y, z;
    uint32_t c;
    read_point(p, i, &x, &y, &z, &c);
    Frag f = project(v, x, y, z, c);
    if (f.visible && f.key < fb[f.pixel]) fb[f.pixel] = f.key;
  }
  return 0;
}

void oracle_clear(uint64_t* fb, uint64_t pixels) {
  for (uint64_t i = 0; i < pixels; ++i) fb[i] = kEmpty;
}

// High-quality splatting pass 2 (Section 2.2). fb is the pass-1 result. Sums and counts are per-pixel
// u64 arrays (separate arrays, not the GPU's packed layout), accumulated (not cleared) here.
// Returns 2 when some pixel's count exceeds 2^24 (the documented sum-capacity limit), else 0.
int oracle_hq_accumulate(const void* points, uint64_t n, const double* M, double near_, double far_,
                         int depth_mode, double metric_scale, int n_ranges, const double* ranges, int W, int H,
                         const uint64_t* fb, uint32_t eps_num, uint32_t eps_den, uint64_t* sum_r, uint64_t* sum_g,
                         uint64_t* sum_b, uint64_t* count) {
  OView v;
  if (!make_view(M, near_, far_, depth_mode, metric_scale, n_ranges, ranges, W, H, &v)) return 1;
  if (eps_den == 0 || depth_mode == 2) return 1;  // the band test needs codes proportional to depth
  // Depth code of the near plane: the offset that turns a linear-mode code back into a depth
  // proportional to w (w * s ~= q + near * s). Metric codes are already proportional to w, so their
  // offset is 0.
  const uint64_t Nq = depth_mode == 0 ? (uint64_t)std::floor(near_ * linear_scale(v)) : 0;
  const unsigned char* p = (const unsigned char*)points;
  int rc = 0;
  for (uint64_t i = 0; i < n; ++i) {
    float x, y, z;
    uint32_t c;
    read_point(p, i, &x, &y, &z, &c);
    Frag f = project(v, x, y, z, c);
    if (!f.visible) continue;
    const uint64_t qmin = fb[f.pixel] >> 24;
    if ((uint64_t)eps_den * (f.q - qmin) <= (uint64_t)eps_num * (qmin + Nq)) {
      sum_r[f.pixel] += c & 0xFF;
      sum_g[f.pixel] += (c >> 8) & 0xFF;
      sum_b[f.pixel] += (c >> 16) & 0xFF;
      count[f.pixel] += 1;
      if (count[f.pixel] > (1ull << 24)) rc = 2;
    }
  }
  return rc;
}

// Basic resolve (Section 2.1, per-pixel shader): RGB of the stored key with alpha 255, or the
// background colour where the pixel is empty.
void oracle_resolve_basic(const uint64_t* fb, uint64_t pixels, uint32_t background, uint32_t* rgba) {
  for (uint64_t i = 0; i < pixels; ++i)
    rgba[i] = fb[i] == kEmpty ? background : ((uint32_t)(fb[i] & 0xFFFFFFu) | 0xFF000000u);
}

// HQ resolve (Section 2.2, third pass): per channel (sum + count / 2) / count, alpha 255; background
// where no fragment contributed.
void oracle_resolve_hq(const uint64_t* sum_r, const uint64_t* sum_g, const uint64_t* sum_b, const uint64_t* count,
                       uint64_t pixels, uint32_t background, uint32_t* rgba) {
  for (uint64_t i = 0; i < pixels; ++i) {
    const uint64_t c = count[i];
    if (c == 0) {
      rgba[i] = background;
      continue;
    }
    const uint32_t r = (uint32_t)((sum_r[i] + c / 2) / c), g = (uint32_t)((sum_g[i] + c / 2) / c),
                   b = (uint32_t)((sum_b[i] + c / 2) / c);
    rgba[i] = r | (g << 8) | (b << 16) | 0xFF000000u;
  }
}

// Brute force for one pixel, structured the other way round: scan every point, keep the smallest key
// among those whose fragment lands on (px, py). O(points) per pixel; for cross-checks on tiny scenes.
uint64_t oracle_bruteforce_pixel(const void* points, uint64_t n, const double* M, double near_, double far_,
                                 int depth_mode, double metric_scale, int n_ranges, const double* ranges, int W,
                                 int H, int px, int py) {
  OView v;
  if (!make_view(M, near_, far_, depth_mode, metric_scale, n_ranges, ranges, W, H, &v)) return 0;
  const unsigned char* p = (const unsigned char*)points;
  uint64_t best = kEmpty;
  const int64_t target = (int64_t)py * W + px;
  for (uint64_t i = 0; i < n; ++i) {
    float x, y, z;
    uint32_t c;
    read_point(p, i, &x, &y, &z, &c);
    Frag f = project(v, x, y, z, c);
    if (f.visible && f.pixel == target && f.key < best) best = f.key;
  }
  return best;
}

}  // extern "C"
