// Seeded synthetic point-cloud generators (input data only).
//
// These stand in for the paper's scanned data sets (Heidentor, Retz, Morro Bay; Table 1), which are
// not available: a uniform cube and a LIDAR-like scene (sin-sum heightfield terrain, axis-aligned box
// buildings, N(0, sigma) coordinate noise, RGB from a height ramp, coherent scan order).
//
// This module holds none of the rasterizer's arithmetic (no projection, no depth quantisation, no
// key packing). Both the oracle tests and the CUDA path consume its output.
//
// Randomness: SplitMix64 used as a counter-based generator. Its published definition advances a
// 64-bit state by the golden-ratio increment 0x9E3779B97F4A7C15 and returns a fixed mixing function
// of the state, so the n-th output of stream `s` is mix(s + (n + 1) * increment). Every random draw
// of point i is addressed by (stream, i, k), which makes the output independent of the thread split.
//
// Point layout: 16 B per point, float x, y, z followed by a little-endian RGBA8 word (byte 0 = R).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// n-th output (n = 0, 1, ...) of the SplitMix64 sequence started from `state`.
inline uint64_t splitmix_at(uint64_t state, uint64_t n) { return mix64(state + (n + 1) * kGolden); }

// Stream key for (seed, tag): the first output of a SplitMix64 sequence seeded with seed ^ tag.
inline uint64_t stream_key(uint64_t seed, uint64_t tag) { return splitmix_at(seed ^ (tag * 0xD1B54A32D192ED03ull), 0); }

// Uniform in [0, 1) from the top 24 bits (exact in float and double).
inline double u24(uint64_t r) { return (double)(r >> 40) * (1.0 / 16777216.0); }
// Uniform in [0, 1) from the top 53 bits.
inline double u53(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

struct Rng {
  uint64_t key;
  uint64_t base;  // point index * draws per point
  inline uint64_t at(uint64_t k) const { return splitmix_at(key, base + k); }
};

struct Point {
  float x, y, z;
  uint32_t rgba;
};
static_assert(sizeof(Point) == 16, "16-byte point");

inline void store_point(void* out, uint64_t i, double x, double y, double z, uint32_t rgba) {
  Point p{(float)x, (float)y, (float)z, rgba};
  std::memcpy((char*)out + i * 16, &p, 16);
}

// Box-Muller: two N(0,1) samples from two uniforms (u1 in (0,1]).
inline void box_muller(uint64_t r1, uint64_t r2, double* a, double* b) {
  const double u1 = 1.0 - u53(r1);  // (0, 1]
  const double u2 = u53(r2);
  const double rad = std::sqrt(-2.0 * std::log(u1));
  const double th = 6.283185307179586 * u2;
  *a = rad * std::cos(th);
  *b = rad * std::sin(th);
}

template <typename F>
void parallel_for(uint64_t n, int nthreads, F&& body) {
  if (nthreads <= 1 || n < (1u << 16)) {
    body(0, n);
    return;
  }
  std::vector<std::thread> th;
  th.reserve(nthreads);
  for (int t = 0; t < nthreads; ++t) {
    uint64_t b = n * (uint64_t)t / (uint64_t)nthreads, e = n * (uint64_t)(t + 1) / (uint64_t)nthreads;
    th.emplace_back([&body, b, e] { body(b, e); });
  }
  for (auto& x : th) x.join();
}

}  // namespace

extern "C" {

typedef struct {
  double x0, x1, y0, y1;          // terrain extent (m), z up
  double amp_scale;               // multiplies the amplitudes 40, 20, 10, 5, 2.5, 1.25 m
  double wavelength_scale;        // multiplies the wavelengths 500, 250, 120, 60, 30, 15 m
  int32_t n_boxes;                // axis-aligned box buildings
  double box_fp_min, box_fp_max;  // footprint side range (m)
  double box_h_min, box_h_max;    // height range (m)
  double noise_sigma;             // N(0, sigma) added to every coordinate (m)
  double street_x, street_y;      // centre of the street-level detail disk
  double street_radius;           // 0 disables street detail
  double street_fraction;         // share of points placed in the street-level detail
  double box_exclusion;           // no building centre within this distance of (street_x, street_y)
} scn_lidar_params;

uint64_t scn_splitmix64_at(uint64_t state, uint64_t n) { return splitmix_at(state, n); }

// Uniform cube [-half, half]^3, RGB = three random bytes, A = 255.
int scn_gen_cube(uint64_t n, uint64_t seed, double half, void* out, int nthreads) {
  if (!out && n) return 1;
  const uint64_t key = stream_key(seed, 1);
  parallel_for(n, nthreads, [&](uint64_t b, uint64_t e) {
    for (uint64_t i = b; i < e; ++i) {
      Rng r{key, i * 4};
      const double x = (u24(r.at(0)) * 2.0 - 1.0) * half;
      const double y = (u24(r.at(1)) * 2.0 - 1.0) * half;
      const double z = (u24(r.at(2)) * 2.0 - 1.0) * half;
      const uint32_t c = (uint32_t)(r.at(3) >> 40);  // 24 random bits: R, G, B
      store_point(out, i, x, y, z, c | 0xFF000000u);
    }
  });
  return 0;
}

namespace {

struct Terrain {
  double A[6], L[6], phi[6], psi[6];
  double height(double x, double y) const {
    double h = 0.0;
    for (int k = 0; k < 6; ++k)
      h += A[k] * std::sin(6.283185307179586 * x / L[k] + phi[k]) * std::sin(6.283185307179586 * y / L[k] + psi[k]);
    return h;
  }
  double amp_sum() const {
    double s = 0;
    for (int k = 0; k < 6; ++k) s += std::fabs(A[k]);
    return s;
  }
};

struct Box {
  double cx, cy, fx, fy, base, h;
  double roof_area() const { return fx * fy; }
  double wall_area() const { return 2.0 * (fx + fy) * h; }
};

// Height ramp: dark blue -> green -> yellow -> red -> white over t in [0, 1].
uint32_t ramp(double t) {
  static const double stops[5][3] = {{0.10, 0.15, 0.45}, {0.15, 0.55, 0.20}, {0.90, 0.85, 0.25}, {0.80, 0.25, 0.15}, {0.97, 0.97, 0.97}};
  if (!(t > 0.0)) t = 0.0;
  if (t > 1.0) t = 1.0;
  const double s = t * 4.0;
  int k = (int)s;
  if (k > 3) k = 3;
  const double f = s - k;
  uint32_t c = 0;
  for (int ch = 0; ch < 3; ++ch) {
    double v = stops[k][ch] * (1.0 - f) + stops[k + 1][ch] * f;
    uint32_t b = (uint32_t)(v * 255.0 + 0.5);
    if (b > 255) b = 255;
    c |= b << (8 * ch);
  }
  return c | 0xFF000000u;
}

}  // namespace

// LIDAR-like scene. Point order: terrain in 1-m strips along y (alternating x direction, like an
// airborne scanner), then building by building (roof, then walls), then street-level detail.
int scn_gen_lidar(uint64_t n, uint64_t seed, const scn_lidar_params* p, void* out, int nthreads) {
  if (!p || (!out && n)) return 1;
  if (!(p->x1 > p->x0) || !(p->y1 > p->y0) || p->n_boxes < 0) return 1;
  static const double A0[6] = {40, 20, 10, 5, 2.5, 1.25};
  static const double L0[6] = {500, 250, 120, 60, 30, 15};
  Terrain T;
  const uint64_t kph = stream_key(seed, 2);
  for (int k = 0; k < 6; ++k) {
    T.A[k] = A0[k] * p->amp_scale;
    T.L[k] = L0[k] * p->wavelength_scale;
    T.phi[k] = 6.283185307179586 * u53(splitmix_at(kph, 2 * k));
    T.psi[k] = 6.283185307179586 * u53(splitmix_at(kph, 2 * k + 1));
  }
  // Buildings.
  std::vector<Box> boxes;
  const uint64_t kbox = stream_key(seed, 3);
  uint64_t draw = 0;
  for (int b = 0; b < p->n_boxes; ++b) {
    Box bx{};
    for (int attempt = 0; attempt < 64; ++attempt) {
      bx.fx = p->box_fp_min + (p->box_fp_max - p->box_fp_min) * u53(splitmix_at(kbox, draw++));
      bx.fy = p->box_fp_min + (p->box_fp_max - p->box_fp_min) * u53(splitmix_at(kbox, draw++));
      bx.h = p->box_h_min + (p->box_h_max - p->box_h_min) * u53(splitmix_at(kbox, draw++));
      bx.cx = p->x0 + bx.fx * 0.5 + (p->x1 - p->x0 - bx.fx) * u53(splitmix_at(kbox, draw++));
      bx.cy = p->y0 + bx.fy * 0.5 + (p->y1 - p->y0 - bx.fy) * u53(splitmix_at(kbox, draw++));
      const double dx = bx.cx - p->street_x, dy = bx.cy - p->street_y;
      if (p->box_exclusion <= 0.0 || std::sqrt(dx * dx + dy * dy) > p->box_exclusion + 0.5 * (bx.fx + bx.fy)) break;
    }
    bx.base = T.height(bx.cx, bx.cy);
    boxes.push_back(bx);
  }
  // Point budget: street share first, the rest proportional to surface area.
  const uint64_t n_street = p->street_radius > 0.0 ? (uint64_t)std::floor((double)n * p->street_fraction) : 0;
  const uint64_t n_surf = n - n_street;
  const double a_terrain = (p->x1 - p->x0) * (p->y1 - p->y0);
  std::vector<double> cum(boxes.size() + 1);
  double a_total = a_terrain;
  cum[0] = a_terrain;
  for (size_t b = 0; b < boxes.size(); ++b) {
    a_total += boxes[b].roof_area() + boxes[b].wall_area();
    cum[b + 1] = a_total;
  }
  std::vector<uint64_t> first(boxes.size() + 2);  // first point index of terrain(0), box b (b+1), street (last)
  first[0] = 0;
  for (size_t b = 0; b <= boxes.size(); ++b) {
    uint64_t c = (b == boxes.size()) ? n_surf : (uint64_t)std::floor((double)n_surf * (cum[b] / a_total));
    first[b + 1] = std::max(c, first[b]);
  }
  const uint64_t n_terrain = first[1];
  const double zmin = -T.amp_sum();
  double zmax = T.amp_sum();
  for (auto& bx : boxes) zmax = std::max(zmax, bx.base + bx.h);
  const uint64_t strips = (uint64_t)std::max(1.0, std::ceil(p->y1 - p->y0));
  const uint64_t kpt = stream_key(seed, 4);
  const double sig = p->noise_sigma;

  parallel_for(n, nthreads, [&](uint64_t b, uint64_t e) {
    size_t box = std::upper_bound(first.begin(), first.end(), b) - first.begin() - 1;
    for (uint64_t i = b; i < e; ++i) {
      while (box + 1 < first.size() && i >= first[box + 1]) ++box;
      Rng r{kpt, i * 8};
      double nx, ny, nz, nw;
      box_muller(r.at(0), r.at(1), &nx, &ny);
      box_muller(r.at(2), r.at(3), &nz, &nw);
      double x, y, z;
      if (i < n_terrain) {
        // Strip k holds the indices i with floor(i * strips / n_terrain) == k.
        const uint64_t k = (uint64_t)(((unsigned __int128)i * strips) / n_terrain);
        const uint64_t f0 = (uint64_t)(((unsigned __int128)k * n_terrain + strips - 1) / strips);
        const uint64_t f1 = (uint64_t)(((unsigned __int128)(k + 1) * n_terrain + strips - 1) / strips);
        const uint64_t m = f1 - f0, j = i - f0;
        double u = ((double)j + u53(r.at(4))) / (double)m;
        if (k & 1) u = 1.0 - u;
        x = p->x0 + u * (p->x1 - p->x0);
        y = p->y0 + std::min((double)k + u53(r.at(5)), p->y1 - p->y0);
        z = T.height(x, y);
      } else if (i < n_surf) {
        const Box& bx = boxes[box - 1];
        const double roof = bx.roof_area(), wall = bx.wall_area();
        const double sel = u53(r.at(4)) * (roof + wall);
        const double a = u53(r.at(5)), c = u53(r.at(6));
        if (sel < roof) {
          x = bx.cx + (a - 0.5) * bx.fx;
          y = bx.cy + (c - 0.5) * bx.fy;
          z = bx.base + bx.h;
        } else {
          // Walls: perimeter parameter s in [0, 2(fx+fy)).
          const double s = (sel - roof) / wall * 2.0 * (bx.fx + bx.fy);
          const double x0 = bx.cx - 0.5 * bx.fx, y0 = bx.cy - 0.5 * bx.fy;
          if (s < bx.fx) { x = x0 + s; y = y0; }
          else if (s < bx.fx + bx.fy) { x = x0 + bx.fx; y = y0 + (s - bx.fx); }
          else if (s < 2 * bx.fx + bx.fy) { x = x0 + bx.fx - (s - bx.fx - bx.fy); y = y0 + bx.fy; }
          else { x = x0; y = y0 + bx.fy - (s - 2 * bx.fx - bx.fy); }
          z = bx.base + a * bx.h;
        }
      } else {
        // Street detail: ground disk around (street_x, street_y) plus small boxes (bollards, posts).
        const double a = u53(r.at(4)), c = u53(r.at(5)), d = u53(r.at(6));
        const double rad = p->street_radius * std::sqrt(a), th = 6.283185307179586 * c;
        x = p->street_x + rad * std::cos(th);
        y = p->street_y + rad * std::sin(th);
        z = T.height(x, y);
        if (d < 0.5) {
          // Snap to one of 64 posts spread over the disk, some of them within centimetres of the centre.
          const uint64_t post = (uint64_t)(d * 128.0);
          const uint64_t pr = splitmix_at(stream_key(seed, 5), post);
          const double pd = 0.05 + (p->street_radius - 0.05) * u24(pr) * u24(pr);
          const double pa = 6.283185307179586 * u53(splitmix_at(stream_key(seed, 6), post));
          const double px = p->street_x + pd * std::cos(pa), py = p->street_y + pd * std::sin(pa);
          const double side = 0.1 + 0.3 * u24(splitmix_at(stream_key(seed, 7), post));
          x = px + (u53(r.at(7)) - 0.5) * side;
          y = py + (c - 0.5) * side;
          z = T.height(px, py) + 2.5 * a;
        }
      }
      x += sig * nx;
      y += sig * ny;
      z += sig * nz;
      store_point(out, i, x, y, z, ramp((z - zmin) / (zmax - zmin)));
    }
  });
  return 0;
}

// Height of the generated terrain at (x, y), for placing cameras (same seed and params as the scene).
double scn_lidar_height(uint64_t seed, const scn_lidar_params* p, double x, double y) {
  static const double A0[6] = {40, 20, 10, 5, 2.5, 1.25};
  static const double L0[6] = {500, 250, 120, 60, 30, 15};
  Terrain T;
  const uint64_t kph = stream_key(seed, 2);
  for (int k = 0; k < 6; ++k) {
    T.A[k] = A0[k] * p->amp_scale;
    T.L[k] = L0[k] * p->wavelength_scale;
    T.phi[k] = 6.283185307179586 * u53(splitmix_at(kph, 2 * k));
    T.psi[k] = 6.283185307179586 * u53(splitmix_at(kph, 2 * k + 1));
  }
  return T.height(x, y);
}

// In-place Fisher-Yates shuffle of n 16-byte points; swap partner of position i drawn from the
// counter stream (seed, tag 8), index i.
int scn_shuffle(void* pts, uint64_t n, uint64_t seed) {
  if (!pts && n) return 1;
  const uint64_t key = stream_key(seed, 8);
  char* base = (char*)pts;
  char tmp[16];
  for (uint64_t i = n; i > 1; --i) {
    const uint64_t j = (uint64_t)(((unsigned __int128)splitmix_at(key, i) * i) >> 64);  // [0, i)
    if (j != i - 1) {
      std::memcpy(tmp, base + (i - 1) * 16, 16);
      std::memcpy(base + (i - 1) * 16, base + j * 16, 16);
      std::memcpy(base + j * 16, tmp, 16);
    }
  }
  return 0;
}

}  // extern "C"
