// Certified single-precision evaluation of the per-point transform.
//
// The definition (Sections 1 and 2.1 of arXiv 1908.02681, as read in include/pcr.h) evaluates clip x,
// clip y and w in FP64, rounds them to float for the pixel mapping, and quantises w to a 40-bit code in
// FP64. GB300 issues FP64 at ~1/80 of its FP32 rate, so this file evaluates each point with FP32 and
// integer arithmetic whose error bounds prove what the FP64 definition gives:
//
//   * depth code: t = S * (w - near) (LINEAR, S = s) or S * w (METRIC, S = metric_scale) is linear in the
//     point, t = sum_j A_j X_j + B with A_j = S * M[3][j]. Each float coordinate X_j = m_j * 2^(e_j - 150)
//     (24-bit integer mantissa m_j, biased exponent e_j), so A_j X_j = m_j * (A_j * 2^(e_j - 150)). A
//     per-view table holds round(A_j * 2^(e - 150) * 2^40) for every sign and exponent (built exactly on
//     the host with 128-bit integers); the point's t * 2^40 is the 96-bit integer sum of three 24x64-bit
//     products and B * 2^40, within 2^-15 of the exact real t. The FP64 definition's own rounding moves t
//     by at most u64 * (5.2 * T_t + 3.1 * S * near), T_t = sum |A_j X_j| + |B|; when the interval of
//     both errors around the integer sum holds no integer, floor(t_FP64) is known exactly.
//   * clip values: each of clip x, clip y, w is evaluated in double-float (matrix entries split into
//     two floats, exact products by fma, error-free two-sums for the large terms), with an error bound
//     of 40 * 2^-48 * T (T = sum of the term magnitudes), which also covers the FP64 definition's three
//     roundings. When that interval holds no float rounding boundary, the float the definition rounds
//     to is known exactly, and the single-precision pixel mapping is then evaluated with the same IEEE
//     operations as the definition.
//
// The pixel is decided in two tiers. Tier 1 evaluates clip x, y, w with plain float fma chains and
// bounds, per point, how far the definition's pixel coordinate fx can be from the float estimate (the
// rounding of the matrix to float, the fma roundings, the definition's own float roundings, the
// approximate reciprocal); when fx and that bound stay inside one pixel, the pixel is known. Points that
// tier 1 cannot decide are queued per warp in shared memory and, 32 at a time, go through tier 2: the
// double-float clip values above, whose float roundings are certified, and the definition's IEEE single
// pixel mapping.
//
// A point whose depth code tier 1 leaves undecided between two neighbours goes to tier 2 too (rare: settling
// it in tier 1 would cost every point extra work). There, pass 1 sends it on only when its smaller candidate
// key could still win its pixel, and pass 2 only when the two candidates give different band answers; a point
// whose cull or pixel tier 2 cannot decide, and those, go through the FP64 definition directly (the arbiter).
// The output is therefore bit-identical to the FP64 definition.
#pragma once

#include <cmath>
#include <cstring>

#include "pcr_kernels.cuh"

namespace pcr {

constexpr int kTableExp = 256;                 // biased float exponents
constexpr int kTableEntries = 2 * kTableExp;   // x sign
constexpr int kFixedFracBits = 40;             // t is held in units of 2^-40

// Per-view constants of the certified evaluation. Passed by value as a __grid_constant__ kernel
// parameter (about 12.8 KB), so concurrent launches with different views share nothing.
struct CertParams {
  // hot scalars first: the per-point loops read them as instruction operands; the table comes last
  float H[3][4], L[3][4];             // float splits of the rows clip x, clip y, w (H: nearest float, L: rest)
  // tier 1 (classify_fast); s = |x| + |y| + |z| of the point, evaluated in float
  float Wr[4];                        // w row, nearest floats of M[3][c]
  float Gx[4], Gy[4];                 // nearest floats of W/2 M[0] + (W/2 - 1/2) M[3], H/2 M[1] + (H/2 - 1/2) M[3]
  float wc, whk, kw, kw3;             // depth window: |w - wc| < whk - kw s certifies near <= w_FP64 < far
  float near_o, far_o;                // RD(near), RU(far): w + dw < near_o or w - dw >= far_o culls
  float ke, ke3, he0;                 // pixel bound: hE = he0 - (ke s + ke3) / w <= 1/2 - E
  float kd, hd0;                      // depth code: hD = hd0 - kd s <= 1/2 - D - 2^-22 + 2^-25
  float Mw, Mw3, MH, MH3, cb, ce;     // cull branch: magnitude sums and the general pixel bound
  float wm, hm;                       // W - 1/2, H - 1/2 (exact)
  float xyz_max;                      // |x| + |y| + |z| below this: table entries usable, values finite
  float kappa;                        // double-float error bound factor (relative to T)
  float t_c1, t_c2;                   // tier-2 bound of t: t_c1 * T_t + t_c2
  float Af[3], Bf;                    // float approximations of A_j and B (for T_t)
  unsigned long long BL;              // tier 1: B * 2^40 = BH * 2^32 + BL, 0 <= BL < 2^32
  long long BH;
  uint32_t B0, B1, B2;                // B * 2^40 as a 96-bit two's-complement integer (low word first)
  int32_t e_max[3];                   // largest biased exponent of x, y, z with a usable table entry
  long long qn_safe, qn_cull, qf_safe, qf_cull;  // depth-cull thresholds in code space
  // approximate (double-float, no arbiter) mode
  float near_h, near_l, far_h, far_l, S_h, S_l;
  int32_t approximate;
  int32_t linear;
  // PIECEWISE depth: the n_pw ranges that meet [near, far) (0: LINEAR or METRIC). Range r has its own depth
  // table (block r of the device table, 3 * kTableEntries entries each), window, code margin and first code.
  int32_t n_pw;
  float pw_wc[kMaxRanges], pw_whk[kMaxRanges], pw_kd[kMaxRanges], pw_hd0[kMaxRanges];
  float pw_start[kMaxRanges];         // ascending split points: range r is the only one whose window may hold
                                      // a w at or above pw_start[r] and below pw_start[r + 1]
  unsigned long long pw_BL[kMaxRanges];  // (B_r + base_r 2^40) = BH 2^32 + BL: the first code folded in
  long long pw_BH[kMaxRanges];
  DevView v;                          // the FP64 definition (for the arbiter)
  long long F[3][kTableEntries];      // t-row fixed-point coefficients, index (sign << 8) | exponent
};

// The first-tier constants of one view (a subset of CertParams with the same field names).
struct HotParams {
  float Wr[4], Gx[4], Gy[4];
  float wc, whk, kw, kw3, near_o, far_o, ke, ke3, he0, kd, hd0, Mw, Mw3, MH, MH3, cb, ce, wm, hm, xyz_max;
  unsigned long long BL;
  long long BH;
  struct {
    int32_t width, height;
  } v;
};

__host__ __device__ inline HotParams hot_params(const CertParams& P) {
  HotParams h;
  for (int c = 0; c < 4; ++c) {
    h.Wr[c] = P.Wr[c];
    h.Gx[c] = P.Gx[c];
    h.Gy[c] = P.Gy[c];
  }
  h.wc = P.wc;
  h.whk = P.whk;
  h.kw = P.kw;
  h.kw3 = P.kw3;
  h.near_o = P.near_o;
  h.far_o = P.far_o;
  h.ke = P.ke;
  h.ke3 = P.ke3;
  h.he0 = P.he0;
  h.kd = P.kd;
  h.hd0 = P.hd0;
  h.Mw = P.Mw;
  h.Mw3 = P.Mw3;
  h.MH = P.MH;
  h.MH3 = P.MH3;
  h.cb = P.cb;
  h.ce = P.ce;
  h.wm = P.wm;
  h.hm = P.hm;
  h.xyz_max = P.xyz_max;
  h.BL = P.BL;
  h.BH = P.BH;
  h.v.width = P.v.width;
  h.v.height = P.v.height;
  return h;
}

// ------------------------------------------------------------------------------------------------ host

namespace host {

// round(a * b * 2^k) as a signed 128-bit integer; false when |result| would reach 2^126.
inline bool fixed_mul(double a, double b, int k, __int128* out) {
  if (a == 0.0 || b == 0.0) {
    *out = 0;
    return true;
  }
  int ea, eb;
  const double fa = std::frexp(a, &ea), fb = std::frexp(b, &eb);
  const long long ma = (long long)std::ldexp(fa, 53), mb = (long long)std::ldexp(fb, 53);  // exact
  const bool neg = (ma < 0) != (mb < 0);
  unsigned __int128 P = (unsigned __int128)(ma < 0 ? -ma : ma) * (unsigned __int128)(mb < 0 ? -mb : mb);
  const int sh = ea - 53 + eb - 53 + k;
  unsigned __int128 mag;
  if (sh >= 0) {
    if (sh >= 126 || (P >> (126 - sh)) != 0) return false;
    mag = P << sh;
  } else if (sh < -120) {
    mag = 0;  // |a b 2^k| < 2^106 * 2^-121: rounds to 0
  } else {
    const unsigned __int128 half = (unsigned __int128)1 << (-sh - 1);
    mag = (P + half) >> (-sh);
  }
  *out = neg ? -(__int128)mag : (__int128)mag;
  return true;
}

inline bool split_float(double m, float* h, float* l) {
  if (!(std::fabs(m) < 3.0e38)) return false;
  if (m != 0.0 && std::fabs(m) < 0x1p-90) return false;  // keep both halves normal floats
  *h = (float)m;
  *l = (float)(m - (double)*h);  // m - h is exact in double
  return true;
}

inline void two_float(double x, float* h, float* l) {
  *h = (float)x;
  *l = (float)(x - (double)*h);
}

// float rounded up / down from a double (directed conversion: the nearest float, moved one step if it
// lies on the wrong side)
inline float f_up(double x) {
  float f = (float)x;
  if ((double)f < x) f = std::nextafter(f, 3.4e38f);
  return f;
}
inline float f_down(double x) {
  float f = (float)x;
  if ((double)f > x) f = std::nextafter(f, -3.4e38f);
  return f;
}

// Constants of tier 1 (classify_fast). Notation: u = 2^-24, v = 2^-53, a = |x| + |y| + |z| of the point, s its
// float evaluation (two roundings: a <= s (1 + 2.0001u)); T_R = sum_c |R_c x_c| + |R_3| for a row R; w*, cx*, cy*
// the exact clip values of the point and w_d, cx_d, cy_d the FP64 definition's.
//   * w estimate wf: float fma chain of the nearest floats of M[3]: |wf - w*| <= 4.0003u T_M3 (one rounding per
//     entry, three fmas); |w_d - w*| <= 3.0001v T_M3. With T_M3 <= Mw s + Mw3, Delta = kw s + kw3 bounds both.
//   * pixel: G = W/2 M[0] + (W/2 - 1/2) M[3] gives G . p = w* (fx* - 1/2), fx* the exact pixel coordinate. The
//     estimate fm = gx * rcp(wf) (gx the fma chain of G's nearest floats; rcp.approx within 2^-23) satisfies
//     |fm - F| <= 3.0002u |fm| + g + b |F|, F = fx* - 1/2, g = 4.001u T_H / wf, b = 4.001u T_M3 / wf,
//     T_H = sum_c (W/2 |M0c| + (W/2 - 1/2) |M3c|) |x_c| + ... The definition's own float roundings (division,
//     fma, product by W) and FP64 errors add |fx_d - fx*| <= 3.0002u (W/2) |nd*| + 2.0001u |fx*| + 2^-22 (the
//     FP64 part is below 2^-28 (g + b (W + 1))). For a point certified inside the image (|fm| < W, and the
//     bound below under 1/2, which gives |F| <= W + 1/2), E = |fx_d - 1/2 - fm| <= u (6.51 M + 3.51) + g +
//     b (M + 1) + 2^-22, M = max(W, H); the same for y with H.
//   * depth code: |t_FP64 - t| <= v (5.2 T_t + 3.1 S near) (see prepare_cert), T_t <= S (M3max a + |M3_3| +
//     near); the fixed-point sum adds < 2^-15.
inline bool tier1_constants(const DevView& v, double S, CertParams* P) {
  const double u = 0x1p-24, v53 = 0x1p-53;
  const double W = v.width, Hd = v.height, M = W > Hd ? W : Hd;
  const double hw = 0.5 * W, hwm = 0.5 * W - 0.5, hh = 0.5 * Hd, hhm = 0.5 * Hd - 0.5;
  const double *m0 = v.m, *m1 = v.m + 4, *m3 = v.m + 8;
  double m3max = 0.0, hmax = 0.0;
  for (int c = 0; c < 4; ++c) {
    const double gx = std::fma(hw, m0[c], hwm * m3[c]), gy = std::fma(hh, m1[c], hhm * m3[c]);
    // every entry a normal float or zero (so its rounding is relative) and finite
    for (double g : {gx, gy, m3[c]})
      if (!(std::fabs(g) < 3.0e38) || (g != 0.0 && std::fabs(g) < 0x1p-100)) return false;
    P->Wr[c] = (float)m3[c];
    P->Gx[c] = (float)gx;
    P->Gy[c] = (float)gy;
    if (c < 3) {
      m3max = std::fmax(m3max, std::fabs(m3[c]));
      hmax = std::fmax(hmax, std::fmax(hw * std::fabs(m0[c]) + hwm * std::fabs(m3[c]),
                                       hh * std::fabs(m1[c]) + hhm * std::fabs(m3[c])));
    }
  }
  const double h3 = std::fmax(hw * std::fabs(m0[3]) + hwm * std::fabs(m3[3]), hh * std::fabs(m1[3]) + hhm * std::fabs(m3[3]));
  // magnitude sums in s: T_M3 <= (Mw s + Mw3) / (1 + 2^-20), T_H <= (MH s + MH3) / (1 + 2^-20)
  const double sl = (1.0 + 2.0001 * u) * (1.0 + 0x1p-20);
  P->Mw = f_up(m3max * sl);
  P->Mw3 = f_up(std::fabs(m3[3]) * (1.0 + 0x1p-20));
  P->MH = f_up(hmax * sl);
  P->MH3 = f_up(h3 * (1.0 + 0x1p-20));
  // depth window: |wf - wc| < RN(whk - kw s) gives |wf - wc| + Delta < wh, with (wc - wh, wc + wh) inside
  // [near_in, far_in]; near_in also keeps t >= 2.5 and far_in keeps t <= 2^40 - 2^25, so the tier-1 code of a
  // point certified visible needs no sign, zero or cap check (t = S (w - near) or S w). The (1 -+ 4u) margins
  // are kept from the FP64 rounding of t near those ends.
  {
    const double t_lo = 2.5, t_hi = 1099511627776.0 - 33554432.0;
    const double w_lo = P->linear ? v.near_ + t_lo / S : t_lo / S;
    const double w_hi = P->linear ? v.near_ + t_hi / S : t_hi / S;
    const double nin = std::fmax(v.near_ * (1.0 + 4.0 * u), w_lo * (1.0 + 4.0 * u));
    const double fin = std::fmin(v.far_ * (1.0 - 4.0 * u), w_hi * (1.0 - 4.0 * u));
    P->kw = f_up(4.0004 * u * (double)P->Mw * (1.0 + 0x1p-20));
    P->kw3 = f_up(4.0004 * u * (double)P->Mw3 * (1.0 + 0x1p-20));
    if (fin > nin) {
      P->wc = (float)(0.5 * (nin + fin));
      const double wh = std::fmin((double)P->wc - nin, fin - (double)P->wc);
      const double whk = (wh - (double)P->kw3) / (1.0 + 2.0001 * u);
      P->whk = whk > 0.0 ? f_down(whk) : 0.0f;  // 0: tier 1 never certifies the depth
    } else {
      P->wc = 0.0f;
      P->whk = 0.0f;
    }
  }
  P->near_o = f_down(v.near_);
  P->far_o = f_up(v.far_);
  // pixel bound of a visible point: (ke s + ke3) / wf >= g + b (M + 1) (with the roundings of s, the fma, the
  // reciprocal and the product folded into the 1 + 2^-19); he0 = 1/2 - u (6.51 M + 3.51) - 2^-22 - 2^-24, the
  // 2^-24 covering the rounding of hE itself (below 2^-25)
  const double cE = 4.001 * u * (1.0 + 0x1p-19);
  P->ke = f_up(cE * ((double)P->MH + (M + 1.0) * (double)P->Mw));
  P->ke3 = f_up(cE * ((double)P->MH3 + (M + 1.0) * (double)P->Mw3));
  P->he0 = f_down(0.5 - u * (6.51 * M + 3.51) - 0x1p-22 - 0x1p-24);
  // cull branch: b and g from the same sums; E <= |fm| (9.67u + 1.3338 b) + 1.335 g + 3.02u max(W/2 - 1/2,
  // H/2 - 1/2) + 2^-21 for any |fm| when b <= 1/4 (the kernel uses 9.8u, 1.35 and ce)
  P->cb = f_up(4.001 * u * (1.0 + 0x1p-19));
  P->ce = f_up(3.05 * u * std::fmax(hwm, hhm) + 0x1p-20);
  P->wm = (float)(W - 0.5);
  P->hm = (float)(Hd - 0.5);
  // depth code: D <= kd s + d0; hD = RN(hd0 - kd s) with hd0 = RD(1/2 - d0 - 2^-22) (the 2^-22 covers the
  // 23-bit truncation of the fraction and the rounding of that fma)
  P->kd = f_up(5.2 * v53 * S * m3max * (1.0 + 2.0001 * u) * (1.0 + 0x1p-18));
  const double nl = P->linear ? v.near_ : 0.0;
  const double d0 = 5.2 * v53 * S * (std::fabs(m3[3]) + nl) * (1.0 + 0x1p-18) + 3.1 * v53 * S * nl + 0x1p-13;
  P->hd0 = f_down(0.5 - d0 - 0x1p-22);
  return true;
}

// The fixed-point depth table of t = S (w - off): F[j][(sign << 8) | e] = round(S M[3][j] 2^(e - 150) 2^40) for
// every sign and biased exponent of coordinate j (0 past the largest usable exponent, which goes to e_max[j]),
// and b = S (M[3][3] - off) 2^40 rounded. False when the scale puts the values out of the representable range.
inline bool build_table(double S, const double* m3, double off, long long (*F)[kTableEntries], int32_t* e_max,
                        __int128* b_out) {
  for (int j = 0; j < 3; ++j) {
    const double a = S * m3[j];
    if (!(std::fabs(a) < 0x1p80)) return false;  // keeps the subnormal shortcut's error below 2^-46
    e_max[j] = 254;
    for (int e = 0; e < kTableExp; ++e) {
      const int ee = e == 0 ? 1 : e;  // subnormals share exponent 1's scale (see the device loop)
      __int128 f;
      const bool ok = e < 255 && fixed_mul(S, m3[j], ee - 150 + kFixedFracBits, &f) &&
                      f < ((__int128)1 << 62) && f > -((__int128)1 << 62);
      if (!ok) {
        if (e_max[j] >= e) e_max[j] = e - 1;
        f = 0;
      }
      F[j][e] = (long long)f;
      F[j][kTableExp + e] = -(long long)f;
    }
    if (e_max[j] < 127) return false;  // coordinates of magnitude 1 would not be usable
  }
  __int128 b, bn = 0;
  if (!fixed_mul(S, m3[3], kFixedFracBits, &b)) return false;
  if (off != 0.0 && !fixed_mul(S, off, kFixedFracBits, &bn)) return false;
  b -= bn;
  if (b >= ((__int128)1 << 94) || b <= -((__int128)1 << 94)) return false;
  *b_out = b;
  return true;
}

// |x| + |y| + |z| below this keeps every coordinate at or below the smallest e_max (table entries usable).
inline float xyz_limit(const int32_t* e_max) {
  int emin = 254;
  for (int j = 0; j < 3; ++j) emin = e_max[j] < emin ? e_max[j] : emin;
  if (emin >= 254) return 3.0e38f;
  return std::ldexp(1.0f, emin - 127 + 1 > 127 ? 127 : emin - 127 + 1);  // 2^(e+1): exponent <= e
}

// Tier-1 constants of one PIECEWISE range r (t = res (w - lo), codes base + floor(t)), for the part
// [lo_e, hi_e) of the range inside [near, far): the depth window (as in tier1_constants, with the range's
// scale and offset), the code margin, the first code. False when the range's codes could reach the cap.
inline bool piecewise_range(double res, double lo, double lo_e, double hi_e, double base, const double* m3,
                            double m3max, CertParams* P, int r) {
  const double u = 0x1p-24, v53 = 0x1p-53;
  const double t_lo = 2.5, t_hi = 1099511627776.0 - 33554432.0;
  const double w_lo = lo + t_lo / res, w_hi = lo + t_hi / res;
  const double nin = std::fmax(lo_e * (1.0 + 4.0 * u), w_lo * (1.0 + 4.0 * u));
  const double fin = std::fmin(hi_e * (1.0 - 4.0 * u), w_hi * (1.0 - 4.0 * u));
  if (fin > nin) {
    P->pw_wc[r] = (float)(0.5 * (nin + fin));
    const double wh = std::fmin((double)P->pw_wc[r] - nin, fin - (double)P->pw_wc[r]);
    const double whk = (wh - (double)P->kw3) / (1.0 + 2.0001 * u);
    P->pw_whk[r] = whk > 0.0 ? f_down(whk) : 0.0f;
  } else {
    P->pw_wc[r] = 0.0f;
    P->pw_whk[r] = 0.0f;
  }
  P->pw_start[r] = f_down(nin);
  // every code of the range stays below the cap: base + (hi_e - lo) res + 2 < 2^40 - 2
  if (!(base + (hi_e - lo) * res * (1.0 + 0x1p-40) + 4.0 < (double)kQMax)) return false;
  P->pw_kd[r] = f_up(5.2 * v53 * res * m3max * (1.0 + 2.0001 * u) * (1.0 + 0x1p-18));
  const double d0 = 5.2 * v53 * res * (std::fabs(m3[3]) + lo) * (1.0 + 0x1p-18) + 3.1 * v53 * res * lo + 0x1p-13;
  P->pw_hd0[r] = f_down(0.5 - d0 - 0x1p-22);
  return true;
}

// Fills P for the view; false when the view is outside the certified evaluation's preconditions (the
// caller then uses the FP64 kernels, which accept every valid view). tables (may be null): receives the
// depth tables, block r for PIECEWISE range r (block 0 is P->F for LINEAR and METRIC).
inline bool prepare_cert(const DevView& v, bool approximate, CertParams* P,
                         long long (*tables)[3][kTableEntries] = nullptr) {
  std::memset(P, 0, sizeof(*P));
  P->v = v;
  P->approximate = approximate ? 1 : 0;
  const bool pw = v.depth_mode == 2;
  if (v.depth_mode != 0 && v.depth_mode != 1 && !pw) return false;
  if (pw && (approximate || !tables)) return false;  // piecewise: the exact transform with device tables only
  P->linear = v.depth_mode != 1;
  if (!(v.near_ >= 0x1p-60) || !(v.far_ < 0x1p100)) return false;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 4; ++c)
      if (!split_float(v.m[4 * r + c], &P->H[r][c], &P->L[r][c])) return false;
  P->kappa = 40.0f * 0x1p-48f * (1.0f + 0x1p-20f);
  const double* m3 = v.m + 8;
  if (pw) {
    // the ranges meeting [near, far), each a LINEAR-like sub-problem with scale res and offset lo
    double m3max = 0.0;
    for (int j = 0; j < 3; ++j) m3max = std::fmax(m3max, std::fabs(m3[j]));
    int n = 0;
    int32_t emin[3] = {254, 254, 254};
    for (int k = 0; k < v.n_ranges; ++k) {
      const double lo_e = std::fmax(v.lo[k], v.near_), hi_e = std::fmin(v.hi[k], v.far_);
      if (!(hi_e > lo_e)) continue;
      const double res = v.res[k];
      if (!(res > 0.0) || !(res < 0x1p100)) return false;
      if (n == 0) {  // the shared tier-1 constants (the scale only enters the window and margin, set per range)
        if (!tier1_constants(v, res, P)) return false;
      }
      int32_t em[3];
      __int128 b;
      if (!build_table(res, m3, v.lo[k], tables[n], em, &b)) return false;
      for (int j = 0; j < 3; ++j) emin[j] = em[j] < emin[j] ? em[j] : emin[j];
      b += (__int128)(unsigned long long)v.base[k] << kFixedFracBits;  // codes of range k start at base_k
      P->pw_BL[n] = (unsigned long long)(uint32_t)(unsigned __int128)b;
      P->pw_BH[n] = (long long)(b >> 32);
      if (!piecewise_range(res, v.lo[k], lo_e, hi_e, v.base[k], m3, m3max, P, n)) return false;
      ++n;
    }
    if (n == 0) return false;  // nothing of [near, far) has a code: every point is culled (FP64 kernels)
    // one range: NaN, so that no w (+inf included) selects the second arm, whose table the kernels do not hold
    if (n == 1) P->pw_start[1] = std::nanf("");
    P->n_pw = n;
    P->xyz_max = xyz_limit(emin);
    std::memcpy(P->F, tables[0], sizeof(P->F));
    P->BL = P->pw_BL[0];
    P->BH = P->pw_BH[0];
    return true;
  }
  const double S = v.scale;
  if (!(S > 0.0) || !(S < 0x1p100)) return false;
  two_float(v.near_, &P->near_h, &P->near_l);
  two_float(v.far_, &P->far_h, &P->far_l);
  two_float(S, &P->S_h, &P->S_l);
  // t = sum_j A_j X_j + B, A_j = S * M[3][j], B = S * (M[3][3] - near) (LINEAR) or S * M[3][3] (METRIC)
  for (int j = 0; j < 3; ++j) P->Af[j] = (float)(S * m3[j]);
  __int128 b;
  if (!build_table(S, m3, P->linear ? v.near_ : 0.0, P->F, P->e_max, &b)) return false;
  const unsigned __int128 bu = (unsigned __int128)b;
  P->B0 = (uint32_t)bu;
  P->B1 = (uint32_t)(bu >> 32);
  P->B2 = (uint32_t)(bu >> 64);
  P->BL = (unsigned long long)(uint32_t)bu;
  P->BH = (long long)(b >> 32);  // arithmetic: b = BH * 2^32 + BL
  const double bd = S * m3[3] - (P->linear ? S * v.near_ : 0.0);
  if (!(std::fabs(bd) < 1e38)) return false;
  P->Bf = (float)bd;
  // |t_FP64 - t| <= u64 * (5.2 * T_t + 3.1 * S * near) (LINEAR; the near term is absent for METRIC);
  // the fixed-point sum adds < 2^-15; 2^-13 covers both that and the float evaluation of the bound.
  const double u64 = 0x1p-53;
  P->t_c1 = (float)(5.2 * u64 * (1.0 + 0x1p-18));
  P->t_c2 = (float)((P->linear ? 3.1 * u64 * S * v.near_ : 0.0) + 0x1p-13);
  if (!tier1_constants(v, S, P)) return false;
  P->xyz_max = xyz_limit(P->e_max);
  // depth-cull thresholds: T_n, T_f are the FP64 codes of the near and far planes (monotone rounding:
  // t > T_n => w >= near, t < T_n => w < near, t < T_f => w < far, t > T_f => w >= far)
  const double Tn = P->linear ? 0.0 : v.near_ * S;
  const double Tf = P->linear ? (v.far_ - v.near_) * S : v.far_ * S;
  if (!(Tf < 0x1p62)) return false;
  P->qn_safe = (long long)std::floor(Tn) + 1;
  P->qn_cull = (long long)std::floor(Tn) - 1;
  P->qf_safe = (long long)std::floor(Tf) - 1;
  P->qf_cull = (long long)std::floor(Tf) + 1;
  if (tables) std::memcpy(tables[0], P->F, sizeof(P->F));
  return true;
}

}  // namespace host

// ---------------------------------------------------------------------------------------------- device

enum : uint32_t { kCulled = 0, kExact = 1, kAmbiguous = 2, kHard = 3, kDefer = 4 };

struct CertFrag {
  uint32_t state;
  uint32_t pixel;
  long long q;  // kExact: the code; kAmbiguous: the smaller of the two candidates
};

__device__ __forceinline__ void two_sum(float a, float b, float* s, float* e) {
  const float x = __fadd_rn(a, b);
  const float bb = __fsub_rn(x, a);
  *e = __fadd_rn(__fsub_rn(a, __fsub_rn(x, bb)), __fsub_rn(b, bb));
  *s = x;
}

// Double-float evaluation of one clip row; returns the float f that the FP64 value rounds to and whether
// that rounding is certified.
__device__ __forceinline__ float df_row(const float* H, const float* L, float x, float y, float z, float kappa,
                                        bool* ok, float* hi_out = nullptr, float* lo_out = nullptr) {
  const float p0 = __fmul_rn(H[0], x), p1 = __fmul_rn(H[1], y), p2 = __fmul_rn(H[2], z);
  const float l0 = __fmaf_rn(L[0], x, __fmaf_rn(H[0], x, -p0));
  const float l1 = __fmaf_rn(L[1], y, __fmaf_rn(H[1], y, -p1));
  const float l2 = __fmaf_rn(L[2], z, __fmaf_rn(H[2], z, -p2));
  float a, ea, b, eb, c, ec;
  two_sum(p0, p1, &a, &ea);
  two_sum(a, p2, &b, &eb);
  two_sum(b, H[3], &c, &ec);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(l0, l1), __fadd_rn(l2, L[3])), __fadd_rn(__fadd_rn(ea, eb), ec));
  const float f = __fadd_rn(c, lo);
  const float r = __fadd_rn(__fsub_rn(c, f), lo);
  const float T = __fadd_rn(__fadd_rn(__fadd_rn(fabsf(p0), fabsf(p1)), fabsf(p2)), fabsf(H[3]));
  const float af = fabsf(f);
  const float ulp_low = __fsub_rn(af, __int_as_float(__float_as_int(af) - 1));
  const float err = __fmaf_rn(kappa, T, __fadd_rn(fabsf(r), 0x1p-126f));
  *ok = err < __fmul_rn(ulp_low, 0.49999994f);
  if (hi_out) {
    *hi_out = c;
    *lo_out = lo;
  }
  return f;
}

__device__ __forceinline__ void mac96(uint32_t m, long long F, uint32_t& a0, uint32_t& a1, uint32_t& a2) {
  const uint32_t flo = (uint32_t)F;
  const int32_t fhi = (int32_t)(F >> 32);
  const unsigned long long p0 = (unsigned long long)m * flo;
  const long long p1 = (long long)(int32_t)m * (long long)fhi;
  asm("add.cc.u32 %0, %0, %3;\n\t"
      "addc.cc.u32 %1, %1, %4;\n\t"
      "addc.u32 %2, %2, 0;\n\t"
      "add.cc.u32 %1, %1, %5;\n\t"
      "addc.u32 %2, %2, %6;"
      : "+r"(a0), "+r"(a1), "+r"(a2)
      : "r"((uint32_t)p0), "r"((uint32_t)(p0 >> 32)), "r"((uint32_t)p1), "r"((uint32_t)((unsigned long long)p1 >> 32)));
}

// Depth row: floor of the fixed-point t (qc) and the top 23 fraction bits as a float in [0, 1).
__device__ __forceinline__ void t_row(const CertParams& P, const long long* __restrict__ F, uint32_t bx, uint32_t by,
                                      uint32_t bz, long long* qc, float* frac) {
  uint32_t a0 = P.B0, a1 = P.B1, a2 = P.B2;
  // a subnormal coordinate takes the implicit bit too; its table entry uses exponent 1's scale, so the
  // product is A * (X + 2^-126 sign(X)): an error below |A| 2^-126, far inside the bound
  mac96((bx & 0x7FFFFFu) | 0x800000u, F[(bx >> 23)], a0, a1, a2);
  mac96((by & 0x7FFFFFu) | 0x800000u, F[kTableEntries + (by >> 23)], a0, a1, a2);
  mac96((bz & 0x7FFFFFu) | 0x800000u, F[2 * kTableEntries + (bz >> 23)], a0, a1, a2);
  *qc = (long long)(int32_t)a2 * 16777216LL + (long long)(a1 >> 8);  // floor(t)
  *frac = __fsub_rn(__uint_as_float(0x3F800000u | (__funnelshift_r(a0, a1, 8) >> 9)), 1.0f);
}

// From the fixed-point t and its error bound D: the candidate codes [qa, qb] (qb = qa or qa + 1) and the
// clip-plane decision. Returns kCulled, kHard, or kExact / kAmbiguous (visible by depth).
__device__ __forceinline__ uint32_t depth_decision(const CertParams& P, long long qc, float frac, float D,
                                                   long long* qa_out) {
  if (D >= 0.5f) return kHard;
  long long qa, qb;
  bool exact;
  if (frac > D && frac < __fsub_rn(1.0f, D)) {
    qa = qb = qc;
    exact = true;
  } else {
    qa = frac < 0.5f ? qc - 1 : qc;
    qb = qa + 1;
    exact = false;
  }
  if (qb <= P.qn_cull || qa >= P.qf_cull) return kCulled;  // culled by the clip planes
  if (qa < P.qn_safe || qb > P.qf_safe) return kHard;
  const long long qmax = (long long)kQMax;
  if (qa >= qmax) exact = true;  // both candidates cap to 2^40 - 2
  *qa_out = qa < qmax ? qa : qmax;
  return exact ? kExact : kAmbiguous;
}

// Tier 2: certified double-float clip values (see the file header). F points at the block's
// shared-memory copy of P.F.
__device__ __forceinline__ CertFrag classify_cert(const CertParams& P, const long long* __restrict__ F, uint4 p) {
  CertFrag out{kCulled, 0u, 0};
  if (P.n_pw) {  // PIECEWISE: a point tier 1 could not decide goes to the FP64 definition
    out.state = kHard;
    return out;
  }
  const uint32_t bx = p.x, by = p.y, bz = p.z;
  const uint32_t ex = (bx >> 23) & 0xFFu, ey = (by >> 23) & 0xFFu, ez = (bz >> 23) & 0xFFu;
  // any NaN or infinite coordinate makes w NaN or infinite in FP64: culled
  if (ex == 0xFFu || ey == 0xFFu || ez == 0xFFu) return out;
  if ((int)ex > P.e_max[0] || (int)ey > P.e_max[1] || (int)ez > P.e_max[2]) {
    out.state = kHard;
    return out;
  }
  long long qc;
  float frac;
  t_row(P, F, bx, by, bz, &qc, &frac);
  const float x = __uint_as_float(bx), y = __uint_as_float(by), z = __uint_as_float(bz);
  const float Tt = __fadd_rn(__fadd_rn(__fadd_rn(fabsf(__fmul_rn(P.Af[0], x)), fabsf(__fmul_rn(P.Af[1], y))),
                                       fabsf(__fmul_rn(P.Af[2], z))), fabsf(P.Bf));
  const float D = __fadd_rn(__fmaf_rn(P.t_c1, Tt, P.t_c2), 0x1p-22f);
  long long qa = 0;
  out.state = depth_decision(P, qc, frac, D, &qa);
  if (out.state == kCulled || out.state == kHard) return out;
  // ---- pixel: certified float roundings of the FP64 clip values, then the definition's float ops
  bool okx, oky, okw;
  const float fw = df_row(P.H[2], P.L[2], x, y, z, P.kappa, &okw);
  const float fcx = df_row(P.H[0], P.L[0], x, y, z, P.kappa, &okx);
  const float fcy = df_row(P.H[1], P.L[1], x, y, z, P.kappa, &oky);
  if (!(okx && oky && okw)) {
    out.state = kHard;
    return out;
  }
  const float fx = __fmul_rn(__fmaf_rn(__fdiv_rn(fcx, fw), 0.5f, 0.5f), P.v.fwidth);
  const float fy = __fmul_rn(__fmaf_rn(__fdiv_rn(fcy, fw), 0.5f, 0.5f), P.v.fheight);
  if (!(fx >= 0.0f && fx < P.v.fwidth && fy >= 0.0f && fy < P.v.fheight)) {
    out.state = kCulled;
    return out;
  }
  out.pixel = (uint32_t)__float2int_rz(fy) * (uint32_t)P.v.width + (uint32_t)__float2int_rz(fx);
  out.q = qa;
  return out;
}

// rcp.approx.ftz.f32: maximum error 1 ulp (relative 2^-23) for normal inputs.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Tier-1 result: state, pixel, and the fixed-point t as three 32-bit words (t * 2^40, low word first).
struct FastFrag {
  uint32_t state;  // kCulled, kExact, kAmbiguous (code undecided between two neighbours), kDefer
  uint32_t pixel;
  uint32_t a0, a1, a2;
};

// Key of the code floor(V / 2^40) (0 <= code < 2^40 - 2): (V >> 16) with the low 24 bits replaced by RGB.
__device__ __forceinline__ unsigned long long key_from_fixed(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t rgba) {
  const uint32_t lo = (__funnelshift_r(a0, a1, 16) & 0xFF000000u) | (rgba & 0xFFFFFFu);
  const uint32_t hi = __funnelshift_r(a1, a2, 16);
  return ((unsigned long long)hi << 32) | lo;
}

__device__ __forceinline__ unsigned long long code_from_fixed(uint32_t a1, uint32_t a2) {
  return ((unsigned long long)(a2 >> 8) << 32) | __funnelshift_r(a1, a2, 8);
}

// Tier 1: the exact depth code from the fixed-point row (two 64-bit multiply-add accumulators), the cull
// from the float w estimate and its bound, and a float pixel estimate with a rigorous per-point bound (the
// constants and their derivation: tier1_constants). All bounds share one magnitude sum s = |x| + |y| + |z|;
// the pixel estimate fm = fx - 1/2 comes from one fma chain per axis (the pixel mapping folded into the clip
// row) and one reciprocal of w. The visible case is decided from predicates without early exits (a
// non-finite coordinate only produces NaN or infinity, which every decision treats as undecided); only a
// point it does not certify takes the branch that tests whether it is certainly culled.
// PP: CertParams (single-view kernels, read from the kernel parameter block) or HotParams (batched
// kernels, which hold one view's first-tier constants in registers); both have the fields used here.
// kPw (PIECEWISE depth, CertParams only): the range whose window certainly holds w gives the table (block r of
// F), the fixed-point offset (with the range's first code folded in: base 2^40 only changes bits 40 and up,
// not the fraction) and the margin. Outside every window: undecided.
// kPw = 1: at most two ranges: a branch on the range (kRange, 0 or 1, selected from w) whose two arms read their
// range's constants at fixed offsets. A warp whose points all lie in one range takes one arm; picking the
// constants per point with selects instead cost 27 more instructions per 32 points and 8 % of pass 1 with the
// paper's nm / um / mm ranges. kPw = 2: any number of ranges, indexed per point.
template <typename PP, int kPw = 0, int kRange = -1>
__device__ __forceinline__ FastFrag classify_fast(const PP& P, const long long* __restrict__ F, uint4 p) {
  const float x = __uint_as_float(p.x), y = __uint_as_float(p.y), z = __uint_as_float(p.z);
  // finite, and inside the exponent range whose table entries exist (else tier 2 decides): the rounded sum of
  // the magnitudes is at least each of them, and NaN or infinity fails the comparison
  const float s = __fadd_rn(__fadd_rn(fabsf(x), fabsf(y)), fabsf(z));
  const bool in_range = s < P.xyz_max;
  // w estimate (fma chain, as the FP64 definition orders it) and the depth window: |w - wc| + Delta < wh
  const float w = __fmaf_rn(P.Wr[2], z, __fmaf_rn(P.Wr[1], y, __fmaf_rn(P.Wr[0], x, P.Wr[3])));
  bool depth_in;
  unsigned long long BL;
  long long BH;
  float kd, hd0;
  int kk = 0;  // PIECEWISE: the range
  (void)kk;
  if constexpr (kPw == 1 && kRange < 0) {
    // one or two ranges (a single range has pw_start[1] = NaN: the second arm is never selected)
    return w >= P.pw_start[1] ? classify_fast<PP, 1, 1>(P, F, p) : classify_fast<PP, 1, 0>(P, F, p);
  }
  if constexpr (kPw == 1) {
    constexpr bool second = kRange == 1;
    kk = second ? 1 : 0;
    depth_in = fabsf(__fsub_rn(w, second ? P.pw_wc[1] : P.pw_wc[0])) <
               __fmaf_rn(-P.kw, s, second ? P.pw_whk[1] : P.pw_whk[0]);
    F += second ? 3 * kTableEntries : 0;
    BL = second ? P.pw_BL[1] : P.pw_BL[0];
    BH = second ? P.pw_BH[1] : P.pw_BH[0];
    kd = second ? P.pw_kd[1] : P.pw_kd[0];
    hd0 = second ? P.pw_hd0[1] : P.pw_hd0[0];
  } else if constexpr (kPw == 2) {
    // the windows are disjoint and ascending: only the last one starting at or below w can hold it
    for (int r = 1; r < P.n_pw; ++r) kk += w >= P.pw_start[r];
    depth_in = fabsf(__fsub_rn(w, P.pw_wc[kk])) < __fmaf_rn(-P.kw, s, P.pw_whk[kk]);
    F += kk * (3 * kTableEntries);
    BL = P.pw_BL[kk];
    BH = P.pw_BH[kk];
    kd = P.pw_kd[kk];
    hd0 = P.pw_hd0[kk];
  } else {
    depth_in = fabsf(__fsub_rn(w, P.wc)) < __fmaf_rn(-P.kw, s, P.whk);
    BL = P.BL;
    BH = P.BH;
    kd = P.kd;
    hd0 = P.hd0;
  }
  // ---- depth code: t * 2^40 = sum m_j F_j + B, accumulated as sum m_j F_lo_j + 2^32 sum m_j F_hi_j
  const long long fx_ = F[p.x >> 23], fy_ = F[kTableEntries + (p.y >> 23)], fz_ = F[2 * kTableEntries + (p.z >> 23)];
  const uint32_t mx = (p.x & 0x7FFFFFu) | 0x800000u, my = (p.y & 0x7FFFFFu) | 0x800000u,
                 mz = (p.z & 0x7FFFFFu) | 0x800000u;
  unsigned long long L = BL;
  L += (unsigned long long)mx * (uint32_t)fx_;
  L += (unsigned long long)my * (uint32_t)fy_;
  L += (unsigned long long)mz * (uint32_t)fz_;
  long long Hh = BH;
  Hh += (long long)(int32_t)mx * (long long)(int32_t)(fx_ >> 32);
  Hh += (long long)(int32_t)my * (long long)(int32_t)(fy_ >> 32);
  Hh += (long long)(int32_t)mz * (long long)(int32_t)(fz_ >> 32);
  FastFrag out;
  out.a0 = (uint32_t)L;
  asm("add.cc.u32 %0, %2, %3;\n\taddc.u32 %1, %4, 0;"
      : "=r"(out.a1), "=r"(out.a2)
      : "r"((uint32_t)(L >> 32)), "r"((uint32_t)Hh), "r"((uint32_t)((unsigned long long)Hh >> 32)));
  const float frac =
      __fsub_rn(__uint_as_float(0x3F800000u | (__funnelshift_r(out.a0, out.a1, 17) & 0x7FFFFFu)), 1.0f);
  // The code is floor(t_FP64) when D < frac_exact < 1 - D, D <= kd s + d0 (the FP64 rounding and the
  // fixed-point sum's error). frac is the fraction truncated to 23 bits (frac <= frac_exact < frac + 2^-23).
  // hD = RN(hd0 - kd s), hd0 = RD(1/2 - d0 - 2^-22), is within 2^-25 of its real value, so |frac - 1/2| < hD
  // (frac - 1/2 is exact) gives D + 2^-22 - 2^-25 < frac and frac + 2^-23 < 1 - D. hD > 1/4 gives D < 1/4:
  // an undecided code still has two usable candidates.
  const float hD = __fmaf_rn(-kd, s, hd0);
  const bool exact = fabsf(__fsub_rn(frac, 0.5f)) < hD;
  const bool amb_ok = hD > 0.25f;

  // ---- pixel estimate: gx = w (fx - 1/2), gy = w (fy - 1/2) up to the rounding bounds; with wf > 0 (depth_in)
  // fm = g * rcp(wf) and the bound hE = RN(he0 - (ke s + ke3) rcp(wf)) <= 1/2 - E - 2^-25
  const float gx = __fmaf_rn(P.Gx[2], z, __fmaf_rn(P.Gx[1], y, __fmaf_rn(P.Gx[0], x, P.Gx[3])));
  const float gy = __fmaf_rn(P.Gy[2], z, __fmaf_rn(P.Gy[1], y, __fmaf_rn(P.Gy[0], x, P.Gy[3])));
  const float r = rcp_approx(w);
  const float fxm = __fmul_rn(gx, r), fym = __fmul_rn(gy, r);
  const float hE = __fmaf_rn(-__fmaf_rn(P.ke, s, P.ke3), r, P.he0);
  // floor of fx = fm + 1/2 via the 1.5 * 2^23 shift: for -1/2 <= fm < 2^22 the sum lies in [2^23, 2^24), where
  // floats are the integers, so g rounds fm to the nearest integer k: floor(fx) unless fx is an integer (then
  // fx - 1 or fx, and |fm - k| = 1/2 fails the test below). Outside that range k, read from the bits, is
  // negative or above 2^22 as an unsigned number: never below the image size.
  const float gxx = __fadd_rn(fxm, 12582912.0f), gyy = __fadd_rn(fym, 12582912.0f);
  const uint32_t kx = (uint32_t)(__float_as_int(gxx) - 0x4B400000), ky = (uint32_t)(__float_as_int(gyy) - 0x4B400000);
  // fm - k = fr - 1/2 (fr = fx - k), exact (k is an integer within 1/2 of fm, both below 2^22)
  const float dx = __fsub_rn(fxm, __fsub_rn(gxx, 12582912.0f)), dy = __fsub_rn(fym, __fsub_rn(gyy, 12582912.0f));
  // E < fr < 1 - E for both axes: |fm - k| < hE < 1/2 - E (hE > 0 also bounds b below 1 / (2M + 1), which the
  // bound E assumes)
  const bool ax_ok = (kx < (uint32_t)P.v.width) & (ky < (uint32_t)P.v.height) & (fabsf(dx) < hE) & (fabsf(dy) < hE);
  uint32_t st;
  if (in_range & depth_in & ax_ok & (exact | amb_ok)) {
    st = exact ? kExact : kAmbiguous;
  } else {
    // Certainly culled? By depth: w_d <= wf + Delta < near, or w_d >= wf - Delta >= far (directed roundings).
    const float dw = __fmaf_rn(P.kw, s, P.kw3);
    const bool depth_out = (__fadd_ru(w, dw) < P.near_o) | (__fsub_rd(w, dw) >= P.far_o);
    // By the pixel, for a point inside the depth window (wf > 0): b, g from the magnitude sums, and the bound
    // E <= |fm| (9.8u + 1.35 b) + 1.35 g + ce, valid at any |fm| while b <= 1/4.
    const float bf = __fmul_rn(__fmul_rn(__fmaf_rn(P.Mw, s, P.Mw3), r), P.cb);
    const float gf = __fmul_rn(__fmul_rn(__fmaf_rn(P.MH, s, P.MH3), r), P.cb);
    const float ea = __fmaf_rn(1.35f, bf, 9.8f * 0x1p-24f), eb = __fmaf_rn(1.35f, gf, P.ce);
    const float ex = __fmaf_rn(fabsf(fxm), ea, eb), ey = __fmaf_rn(fabsf(fym), ea, eb);
    // fx_d < 0 when fm + 1/2 + E < 0; fx_d >= W when fm + 1/2 - E >= W (for finite bounds: an overflow leaves
    // the point to tier 2)
    const bool ax_out = (fxm < -__fadd_ru(0.5f, ex)) | (fxm >= __fadd_ru(P.wm, ex)) | (fym < -__fadd_ru(0.5f, ey)) |
                        (fym >= __fadd_ru(P.hm, ey));
    const bool e_finite = __fadd_rn(ex, ey) < 3.0e38f;
    st = in_range & (depth_out | (depth_in & (bf <= 0.25f) & e_finite & ax_out)) ? kCulled : kDefer;
  }
  out.state = st;
  out.pixel = ky * (uint32_t)P.v.width + kx;
  return out;
}

// Approximate mode (precision study): double-float clip values and depth, no certification, no arbiter.
__device__ __forceinline__ CertFrag classify_df(const CertParams& P, uint4 p) {
  CertFrag out{kCulled, 0u, 0};
  const float x = __uint_as_float(p.x), y = __uint_as_float(p.y), z = __uint_as_float(p.z);
  if (((p.x >> 23) & 0xFFu) == 0xFFu || ((p.y >> 23) & 0xFFu) == 0xFFu || ((p.z >> 23) & 0xFFu) == 0xFFu) return out;
  bool ok;
  float wh, wl, ch, cl;
  const float fw = df_row(P.H[2], P.L[2], x, y, z, P.kappa, &ok, &wh, &wl);
  // w - near and w - far in double-float: visible iff w >= near and w < far
  float dh, dl, gh, gl;
  two_sum(wh, -P.near_h, &dh, &dl);
  dl = __fadd_rn(dl, __fsub_rn(wl, P.near_l));
  two_sum(wh, -P.far_h, &gh, &gl);
  gl = __fadd_rn(gl, __fsub_rn(wl, P.far_l));
  const float dn = __fadd_rn(dh, dl), df = __fadd_rn(gh, gl);
  if (!(dn >= 0.0f && df < 0.0f)) return out;
  const float fcx = df_row(P.H[0], P.L[0], x, y, z, P.kappa, &ok, &ch, &cl);
  const float fcy = df_row(P.H[1], P.L[1], x, y, z, P.kappa, &ok);
  const float fx = __fmul_rn(__fmaf_rn(__fdiv_rn(fcx, fw), 0.5f, 0.5f), P.v.fwidth);
  const float fy = __fmul_rn(__fmaf_rn(__fdiv_rn(fcy, fw), 0.5f, 0.5f), P.v.fheight);
  if (!(fx >= 0.0f && fx < P.v.fwidth && fy >= 0.0f && fy < P.v.fheight)) return out;
  out.pixel = (uint32_t)__float2int_rz(fy) * (uint32_t)P.v.width + (uint32_t)__float2int_rz(fx);
  // t = (w - near) * S or w * S, double-float product
  float th, tl;
  {
    const float ah = P.linear ? dh : wh;
    const float al = P.linear ? dl : wl;
    float sh, sl;
    two_sum(ah, al, &sh, &sl);  // renormalise
    th = __fmul_rn(sh, P.S_h);
    tl = __fadd_rn(__fmaf_rn(sh, P.S_h, -th), __fmaf_rn(sh, P.S_l, __fmul_rn(sl, P.S_h)));
  }
  const float fl = floorf(th);
  const float rem = __fadd_rn(__fsub_rn(th, fl), tl);
  long long q = (long long)fl + (long long)floorf(rem);
  if (q < 0) q = 0;
  const long long qmax = (long long)kQMax;
  out.q = q < qmax ? q : qmax;
  out.state = kExact;
  (void)ch;
  (void)cl;
  return out;
}

__device__ __forceinline__ void load_table(const CertParams& P, long long* sF) {
  const long long* src = &P.F[0][0];
  for (int i = threadIdx.x; i < 3 * kTableEntries; i += blockDim.x) sF[i] = src[i];
  __syncthreads();
}

// The same table from a device-memory copy (coalesced loads; from the kernel parameter block, every lane
// reading its own address, the copy took ~14 us per launch). table == null: from the parameter block.
__device__ __forceinline__ void load_table(const CertParams& P, const long long* __restrict__ table, long long* sF) {
  if (table == nullptr) {
    load_table(P, sF);
    return;
  }
  for (int i = threadIdx.x; i < 3 * kTableEntries; i += blockDim.x) sF[i] = table[i];
  __syncthreads();
}

// Pass 1 at 64 registers and 4 blocks per SM: no spills, and the fastest measured shape (6 blocks at 40
// registers spills and runs 9 % slower on a 100M-point frame).
#ifndef PCR_CERT_MIN_BLOCKS
#define PCR_CERT_MIN_BLOCKS 4
#endif
// The double-float mode (no table, no deferral queue) fits 40 registers without spills and runs fastest at 6.
#ifndef PCR_CERT_APPROX_MIN_BLOCKS
#define PCR_CERT_APPROX_MIN_BLOCKS 6
#endif
#ifndef PCR_CERT_THREADS
#define PCR_CERT_THREADS 256
#endif
constexpr int kCertThreads = PCR_CERT_THREADS;
constexpr int kCertWarps = kCertThreads / 32;
constexpr int kQueue = 64;  // per-warp deferral queue (points), >= 2 * 32 - 1

// ------------------------------------------------------------------------------ point staging (bulk copy)
//
// The single-view passes stream the points through shared memory. Each warp owns a two-stage ring of
// tiles of kTile points (two per lane) and takes the tiles g, g + G, g + 2G, ... of the cloud (g = its
// warp index in the grid, G = warps in the grid). The bulk-copy engine (cp.async.bulk, completion counted
// in bytes on one mbarrier per stage) fills one stage while the warp classifies the points of the other,
// so the warp waits on shared memory instead of on HBM latency. Every wait is bounded; a wait that gives
// up sets the timeout bit of the framebuffer's status word and the warp stops.
constexpr int kTile = 64;
constexpr uint32_t kSpinLimit = 1u << 18;  // try_wait rounds; a round that fails suspends ~3.9 us: about 1 s

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ring_init(uint64_t* bar) {  // one lane; then __syncwarp
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar + 1)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Copies tile t (if it exists) into dst; one lane. A partial last tile copies only its points (16 B each,
// so size and both addresses stay multiples of 16 bytes).
__device__ __forceinline__ void ring_issue(uint4* dst, uint64_t* bar, const uint4* pts, uint64_t n, uint64_t t) {
  const uint64_t first = t * kTile;
  if (first >= n) return;
  const uint64_t left = n - first;
  const uint32_t bytes = (left < (uint64_t)kTile ? (uint32_t)left : (uint32_t)kTile) * 16u;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(pts + first), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ bool ring_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}

// Bounded wait for the completion of the stage's phase with this parity; the same answer in every lane.
__device__ __forceinline__ bool ring_wait(uint64_t* bar, uint32_t parity, uint32_t limit = kSpinLimit) {
  bool ok = ring_try_wait(bar, parity);
  if (__any_sync(0xFFFFFFFFu, !ok)) {
    for (uint32_t spin = 0; !ok && spin < limit; ++spin) ok = ring_try_wait(bar, parity);
    return !__any_sync(0xFFFFFFFFu, !ok);
  }
  return true;
}

// Check of the timeout path: one warp waits, with the passes' ring_wait, on a stage barrier that no copy
// will ever complete (nothing is in flight), gives up after `limit` rounds and sets the timeout bit.
__global__ void k_wait_check(uint32_t* __restrict__ status, uint32_t limit) {
  __shared__ __align__(8) uint64_t bar[2];
  if (threadIdx.x == 0) ring_init(bar);
  __syncwarp();
  if (!ring_wait(&bar[0], 0u, limit) && threadIdx.x == 0) atomicOr(status, kStatusTimeout);
}

// Runs body(p0, valid0, p1, valid1, tile) on every tile of the warp: the lane's two points of the tile (points
// tile * 64 + lane and tile * 64 + 32 + lane); all 32 lanes call body together (body may use warp
// collectives). Returns false when a bounded wait gave up.
template <typename Body>
__device__ __forceinline__ bool stream_ring(const uint4* __restrict__ pts, uint64_t n, uint4 (*ring)[kTile],
                                            uint64_t* bar, uint32_t lane, Body&& body) {
  const uint64_t n_tiles = (n + kTile - 1) / kTile;
  const uint64_t G = (uint64_t)gridDim.x * kCertWarps;
  const uint64_t g = (uint64_t)blockIdx.x * kCertWarps + (threadIdx.x >> 5);
  if (lane == 0) {
    ring_issue(ring[0], &bar[0], pts, n, g);
    ring_issue(ring[1], &bar[1], pts, n, g + G);
  }
  uint32_t s = 0, phases = 0;  // stage of the next tile; bit k = parity of stage k's next phase
  for (uint64_t t = g; t < n_tiles; t += G) {
    if (!ring_wait(&bar[s], (phases >> s) & 1u)) {
      // the other stage's copy (tile t + G) may still be in flight: let it land before the block exits
      if (t + G < n_tiles) ring_wait(&bar[s ^ 1u], (phases >> (s ^ 1u)) & 1u);
      return false;
    }
    const uint64_t left = n - t * kTile;
    const uint32_t cnt = left < (uint64_t)kTile ? (uint32_t)left : (uint32_t)kTile;
    const uint4 p0 = ring[s][lane];
    const uint4 p1 = ring[s][lane + 32];
    __syncwarp();
    if (lane == 0) {  // the stage is free again: refill it with the warp's tile after next
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      ring_issue(ring[s], &bar[s], pts, n, t + 2 * G);
    }
    phases ^= 1u << s;
    s ^= 1u;
    body(p0, lane < cnt, p1, lane + 32u < cnt, t);
  }
  return true;
}

// The same tiles in the same order, loaded by the warp itself (16-byte loads, not allocated in L1), one tile
// ahead: the two points of the warp's next tile are requested before the current tile is classified, so their
// memory latency overlaps the classification. Full tiles take no bounds checks; the partial last tile (if any)
// goes to the warp whose turn it is. No waits: always returns true. Measured on the 100M-point LIDAR frame it
// issues fewer instructions per point than the ring (no barrier, copy or phase bookkeeping per tile) and runs
// pass 1 in 0.58 ms against 0.71 ms.
template <typename Body>
__device__ __forceinline__ bool stream_direct(const uint4* __restrict__ pts, uint64_t n, uint32_t lane, Body&& body) {
  const uint64_t n_full = n / kTile;
  const uint64_t G = (uint64_t)gridDim.x * kCertWarps;
  uint64_t t = (uint64_t)blockIdx.x * kCertWarps + (threadIdx.x >> 5);
  const uint4* p = pts + t * kTile + lane;
  const uint64_t step = G * kTile;
  uint4 a0 = make_uint4(0u, 0u, 0u, 0u), a1 = a0;
  if (t < n_full) {
    a0 = ld_stream16(p);
    a1 = ld_stream16(p + 32);
  }
#pragma unroll 1
  for (; t < n_full; t += G) {
    const uint4 c0 = a0, c1 = a1;
    if (t + G < n_full) {
      p += step;
      a0 = ld_stream16(p);
      a1 = ld_stream16(p + 32);
    }
    body(c0, true, c1, true, t);
  }
  const uint32_t rem = (uint32_t)(n - n_full * kTile);
  if (t == n_full && rem != 0u) {
    const uint4* b = pts + n_full * kTile;
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    const uint4 c0 = lane < rem ? ld_stream16(b + lane) : z;
    const uint4 c1 = lane + 32u < rem ? ld_stream16(b + lane + 32) : z;
    body(c0, lane < rem, c1, lane + 32u < rem, n_full);
  }
  return true;
}

// Point staging of the certified passes: kRing selects the bulk-copy rings (stream_ring), else direct loads
// (stream_direct). A tuning choice (pcr_tuning.staging); both give the same results.
template <bool kRing, typename Body>
__device__ __forceinline__ bool stream_tiles(const uint4* __restrict__ pts, uint64_t n, uint4 (*ring)[kTile],
                                             uint64_t* bar, uint32_t lane, Body&& body) {
  if constexpr (kRing)
    return stream_ring(pts, n, ring, bar, lane, body);
  else
    return stream_direct(pts, n, lane, body);
}

// Pass-1 handling of a tier-2 result: returns true when the point still has to go to the FP64 arbiter.
__device__ __forceinline__ bool raster_commit(const CertFrag& f, uint32_t rgba, unsigned long long* keys) {
  if (f.state == kExact) {
    atomicMin(keys + f.pixel, make_key((unsigned long long)f.q, rgba));
    return false;
  }
  if (f.state == kAmbiguous)  // the smaller candidate cannot win when not below the stored key
    return make_key((unsigned long long)f.q, rgba) < keys[f.pixel];
  return f.state == kHard;
}

// Tier 2 + arbiter for one deferred point (pass 1). Kept out of line: it runs for a small fraction of the
// points, and inlining it would raise the register count of the main loop.
__device__ __noinline__ void raster_deferred(const CertParams& P, const long long* sF, uint4 p,
                                             unsigned long long* keys, unsigned* c_fp64) {
  const CertFrag f = classify_cert(P, sF, p);
  if (raster_commit(f, p.w, keys)) {
    ++*c_fp64;
    uint32_t pix;
    unsigned long long q;
    if (project_fp64(P.v, __uint_as_float(p.x), __uint_as_float(p.y), __uint_as_float(p.z), &pix, &q))
      atomicMin(keys + pix, make_key(q, p.w));
  }
}

// The key a pixel holds, read through L1 (ld.global.ca). Pass 1 reads it before its atomic and skips the atomic
// when the fragment's key is not below it: a stored key only decreases, so such a key can never become the
// minimum, and the result is the same. On a coherent point order, where consecutive points share pixels, this
// halves the atomic minima (same-address atomics serialise in L2). L1 is not coherent with the other SMs'
// atomics within a launch, so pass 1 may read an older key; an older key is never smaller, so the skip (and
// the band record, see BandMask) only becomes more permissive and the atomic still decides. Pass 2 reads the
// final minima, which no launch changes while it runs (a launch starts with the previous launches' writes
// visible). Measured in the 100M-point frame against L2-only reads on the same GPU: pass 1 1.6 % and pass 2
// 2.8 % faster in scan order, pass 2 5.2 % faster shuffled. kL1 = false reads from L2 only: the PIECEWISE
// pass 1, whose per-range tables take more of the shared memory that L1 shares, is 1 % faster that way.
template <bool kL1 = true>
__device__ __forceinline__ unsigned long long stored_key(const unsigned long long* keys, uint32_t pix) {
  if constexpr (kL1) return __ldca(keys + pix);
  return __ldcg(keys + pix);
}

// Lanes a lane may merge with when merging is limited to aligned groups of `width` lanes (8, 16 or 32).
__device__ __forceinline__ uint32_t merge_segment(uint32_t lane, uint32_t width) {
  return width >= 32u ? 0xFFFFFFFFu : ((1u << width) - 1u) << (lane & ~(width - 1u));
}

// Commits one key per lane (has = true) with one atomic minimum per distinct pixel of each lane segment
// (seg: merge_segment): lanes whose fragments land on the same pixel are grouped (match.any) and their
// smallest key found with two 32-bit reductions (high word, then low word among the lanes holding the
// smallest high word). All 32 lanes must call it.
template <bool kMerge>
__device__ __forceinline__ void commit_min(bool has, uint32_t pix, unsigned long long key, unsigned long long* keys,
                                           uint32_t lane, uint32_t seg = 0xFFFFFFFFu) {
  if (!kMerge) {
    if (has) atomicMin(keys + pix, key);
    return;
  }
  const unsigned act = __ballot_sync(0xFFFFFFFFu, has);
  if (has) {
    const unsigned grp = __match_any_sync(act, pix) & seg;
    const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
    const unsigned mhi = __reduce_min_sync(grp, hi);
    const unsigned mlo = __reduce_min_sync(grp, hi == mhi ? lo : 0xFFFFFFFFu);
    if ((grp & ((1u << lane) - 1u)) == 0u) atomicMin(keys + pix, ((unsigned long long)mhi << 32) | mlo);
  }
}

// Appends the deferring lanes' points to the warp's shared-memory queue; when 32 are queued, each lane
// takes one and runs `handle` on it (all 32 lanes converged). qn is warp-uniform.
template <typename H>
__device__ __forceinline__ void defer_points(bool defer, const uint4& p, uint4* q, uint32_t& qn, uint32_t lane,
                                             H&& handle) {
  const unsigned m = __ballot_sync(0xFFFFFFFFu, defer);
  if (m == 0u) return;
  if (defer) q[qn + __popc(m & ((1u << lane) - 1u))] = p;
  qn += __popc(m);
  __syncwarp();
  if (qn >= 32u) {
    qn -= 32u;
    const uint4 d = q[qn + lane];
    __syncwarp();
    handle(d);
  }
}

// Pass 1 (Section 2.1) with the certified transform. Tier 1 handles nearly every point; the others are
// queued per warp in shared memory and handled 32 at a time by tier 2 and the FP64 arbiter. The points
// arrive through stream_tiles (direct loads or bulk-copy rings). kPw > 0: PIECEWISE depth (see classify_fast),
// the ranges' tables in dynamic shared memory (P.n_pw blocks of 3 * kTableEntries entries, from the device table).
// kBand: also writes the band mask for pass 2 (band.mask: two words per tile of 64 points, bit lane of word
// 2 tile + k for point 64 tile + 32 k + lane): the bit is clear when the point is culled, or when its key is
// certainly outside the final band of eps = eps_num / eps_den = E + f (E integer, 0 <= f < 1). The test takes
// the keys' high words only, kh = key >> 32 and sh = sk >> 32 (sk the key its pixel held when it was read), in
// integers: kh >= sh (1 + E) + floor(sh mf / 2^32) + C + 1, with mf >= f 2^32 and C 2^8 >= 255 (1 + eps) +
// eps Nq + 1. Since q = key >> 24 >= kh 2^8 and qs = sk >> 24 <= sh 2^8 + 255, that gives q > qs (1 + eps) +
// eps Nq, i.e. eps_den (q - qs) > eps_num (qs + Nq). The pixel's final minimum is at most qs (a stored key only
// decreases), so q is beyond the final band too. A point the test cannot place keeps its bit (pass 2 decides).
struct BandMask {
  uint32_t* mask;
  uint32_t e1p, mf;      // 1 + E; ceil(f 2^32)
  unsigned long long c1; // C + 1
};

inline BandMask band_mask(uint32_t* mask, uint32_t eps_num, uint32_t eps_den, unsigned long long nq) {
  BandMask b{mask, 1u + eps_num / eps_den, 0u, 0ull};
  const unsigned __int128 fr = (((unsigned __int128)(eps_num % eps_den)) << 32) + eps_den - 1;  // ceil
  const unsigned long long mf = (unsigned long long)(fr / eps_den);
  if (mf >> 32) {  // f 2^32 rounded up to 2^32: one more in the integer part
    b.e1p += 1u;
  } else {
    b.mf = (uint32_t)mf;
  }
  // C = ceil((255 (den + num) + num Nq + den) / (256 den))
  const unsigned __int128 numer = (unsigned __int128)255 * ((unsigned __int128)eps_den + eps_num) +
                                  (unsigned __int128)eps_num * nq + eps_den;
  const unsigned __int128 den = (unsigned __int128)256 * eps_den;
  const unsigned __int128 c = (numer + den - 1) / den;
  if (b.e1p > (1u << 24) || c > ((unsigned __int128)1 << 56)) {
    // an eps this large leaves no code beyond the band worth dropping: the record keeps every point (a bound of
    // 2^62 exceeds every high word, and the sum cannot wrap)
    b.e1p = 0u;
    b.mf = 0u;
    b.c1 = 1ull << 62;
  } else {
    b.c1 = (unsigned long long)c + 1ull;  // sh e1p + c1 + umulhi < 2^56 + 2^56 + 2^32: no wrap
  }
  return b;
}

template <bool kApprox, bool kMerge, bool kStats, bool kRing, int kPw, bool kBand = false>
__global__ void __launch_bounds__(kCertThreads, kApprox ? PCR_CERT_APPROX_MIN_BLOCKS : PCR_CERT_MIN_BLOCKS) k_raster_cert(
    const uint4* __restrict__ pts, uint64_t n, const __grid_constant__ CertParams P,
    unsigned long long* __restrict__ keys, unsigned long long* __restrict__ stats, uint32_t* __restrict__ status,
    const long long* __restrict__ table, BandMask band = BandMask{nullptr, 1u, 0u, 0ull}) {
  __shared__ long long sF_static[kPw ? 1 : 3 * kTableEntries];
  extern __shared__ __align__(16) long long sF_dynamic[];
  __shared__ uint4 queue[kCertWarps][kQueue];
  __shared__ __align__(128) uint4 ring[kCertWarps][2][kTile];
  __shared__ __align__(8) uint64_t bars[kCertWarps][2];
  long long* const sF = kPw ? sF_dynamic : sF_static;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  if (kRing && lane == 0) ring_init(bars[warp]);
  __syncwarp();
  if constexpr (kPw) {
    for (int i = threadIdx.x; i < P.n_pw * 3 * kTableEntries; i += blockDim.x) sF[i] = table[i];
    __syncthreads();
  } else if (!kApprox) {
    load_table(P, table, sF);
  }
  uint4* q = queue[warp];
  uint32_t qn = 0;
  unsigned c_exact = 0, c_amb = 0, c_fp64 = 0, c_defer = 0;
  // Per point: tier 1 (or the double-float evaluation), the atomic minimum of a decided fragment whose key
  // is below the stored key, then the deferral of a point tier 1 could not decide. Committing before the
  // deferral keeps the fragment out of the registers that live across the out-of-line tier-2 call.
  // Returns whether pass 2 may need the point (kBand).
  auto point = [&](const uint4& p, bool valid) -> bool {
    bool defer = false, has = false;
    uint32_t pix = 0;
    unsigned long long key = 0;
    if (valid) {
      if (kApprox) {
        const CertFrag f = classify_df(P, p);
        has = f.state == kExact;
        pix = f.pixel;
        key = make_key((unsigned long long)f.q, p.w);
      } else {
        const FastFrag f = classify_fast<CertParams, kPw>(P, sF, p);
        pix = f.pixel;
        key = key_from_fixed(f.a0, f.a1, f.a2, p.w);
        has = f.state == kExact;
        // an undecided pixel, or a code undecided between two neighbours (rare: settling it here would cost
        // every point a predicated key read), goes to tier 2
        defer = f.state >= kAmbiguous;
        if (kStats) c_amb += f.state == kAmbiguous;
        if (kStats) {
          c_exact += has;
          c_defer += defer;
        }
      }
    }
    const unsigned long long sk = has ? stored_key<kPw == 0>(keys, pix) : 0ull;
    commit_min<kMerge>(has && key < sk, pix, key, keys, lane);
    bool need = defer;
    if constexpr (kBand) {
      const uint32_t kh = (uint32_t)(key >> 32), sh = (uint32_t)(sk >> 32);
      const unsigned long long bound = (unsigned long long)sh * band.e1p + band.c1 + __umulhi(sh, band.mf);
      need |= has && !(kh >= bound);
    }
    if (!kApprox)
      defer_points(defer, p, q, qn, lane, [&](const uint4& d) { raster_deferred(P, sF, d, keys, &c_fp64); });
    return need;
  };
  const bool done = stream_tiles<kRing>(pts, n, ring[warp], bars[warp], lane,
                                 [&](const uint4& p0, bool v0, const uint4& p1, bool v1, uint64_t tile) {
                                   const bool n0 = point(p0, v0);
                                   const bool n1 = point(p1, v1);
                                   if constexpr (kBand) {
                                     const unsigned m0 = __ballot_sync(0xFFFFFFFFu, n0);
                                     const unsigned m1 = __ballot_sync(0xFFFFFFFFu, n1);
                                     if (lane == 0) reinterpret_cast<uint2*>(band.mask)[tile] = make_uint2(m0, m1);
                                   }
                                 });
  if (!done && lane == 0) atomicOr(status, kStatusTimeout);
  if (!kApprox && lane < qn) raster_deferred(P, sF, q[lane], keys, &c_fp64);
  if (kStats) {
    atomicAdd(stats + 0, (unsigned long long)c_exact);
    atomicAdd(stats + 1, (unsigned long long)c_amb);
    atomicAdd(stats + 2, (unsigned long long)c_fp64);
    atomicAdd(stats + 3, (unsigned long long)c_defer);
  }
}

// Pass-2 decision for a tier-2 result: accept, reject, or (return true) send to the arbiter.
__device__ __forceinline__ bool hq_decide(const CertParams& P, const CertFrag& f, const unsigned long long* keys,
                                          uint32_t eps_num, uint32_t eps_den, bool* accept) {
  *accept = false;
  if (f.state == kHard) return true;
  if (f.state != kExact && f.state != kAmbiguous) return false;
  const unsigned long long qmin = keys[f.pixel] >> 24;
  const unsigned long long q = (unsigned long long)f.q;
  *accept = in_band(q, qmin, P.v.nq, eps_num, eps_den);
  if (f.state == kAmbiguous) {
    const unsigned long long q2 = q + 1 < kQMax ? q + 1 : kQMax;
    if (*accept != in_band(q2, qmin, P.v.nq, eps_num, eps_den)) {
      *accept = false;
      return true;
    }
  }
  return false;
}

__device__ __forceinline__ void hq_add(unsigned long long* accum, uint32_t pix, uint32_t rgba) {
  atomicAdd(accum + 2 * (uint64_t)pix, hq_rg(rgba));
  atomicAdd(accum + 2 * (uint64_t)pix + 1, hq_bc(rgba));
}

// Adds the colours of the accepted fragments with one pair of atomics per distinct pixel of each lane segment
// (per-channel sums: at most 32 * 255, no carry between the packed fields). All lanes must call it.
template <bool kMerge>
__device__ __forceinline__ void commit_add(bool add, uint32_t pix, uint32_t rgba, unsigned long long* accum,
                                           uint32_t lane, uint32_t seg = 0xFFFFFFFFu) {
  if (!kMerge) {
    if (add) hq_add(accum, pix, rgba);
    return;
  }
  const unsigned act = __ballot_sync(0xFFFFFFFFu, add);
  if (add) {
    const unsigned grp = __match_any_sync(act, pix) & seg;
    const unsigned r = __reduce_add_sync(grp, rgba & 0xFFu);
    const unsigned g = __reduce_add_sync(grp, (rgba >> 8) & 0xFFu);
    const unsigned b = __reduce_add_sync(grp, (rgba >> 16) & 0xFFu);
    if ((grp & ((1u << lane) - 1u)) == 0u) {
      atomicAdd(accum + 2 * (uint64_t)pix, (unsigned long long)r | ((unsigned long long)g << 32));
      atomicAdd(accum + 2 * (uint64_t)pix + 1, (unsigned long long)b | ((unsigned long long)__popc(grp) << 32));
    }
  }
}

// Adds the colours of the accepted fragments, merged in lane pairs: lanes 2k and 2k + 1 hold consecutive points
// (a warp's tiles and candidate batches are in point order), so on a scan-ordered cloud they often add to one
// pixel; lane 2k then adds both colours with one pair of atomics and lane 2k + 1 none (per-channel sums of two
// fragments: no carry between the packed fields). Three shuffles per point. Measured in the 100M-point frame
// on one GPU: pass 2 3.5 % faster in scan order and 3.9 % shuffled than one pair of atomics per fragment;
// merging groups of 4 or 8 lanes the same way (64-bit sums shuffled) was slower. All lanes must call it.
__device__ __forceinline__ void commit_add_pairs(bool add, uint32_t pix, uint32_t rgba, unsigned long long* accum,
                                                 uint32_t lane) {
  const uint32_t key = add ? pix : 0xFFFFFFFFu;  // pixel indices stay below 2^28
  const uint32_t key_next = __shfl_down_sync(0xFFFFFFFFu, key, 1);
  const uint32_t key_prev = __shfl_up_sync(0xFFFFFFFFu, key, 1);
  const uint32_t rgba_next = __shfl_down_sync(0xFFFFFFFFu, rgba, 1);
  const bool even = (lane & 1u) == 0u;
  if (!add || (!even && key_prev == key)) return;  // nothing to add, or added by lane 2k
  unsigned long long rg = hq_rg(rgba), bc = hq_bc(rgba);
  if (even && key_next == key) {
    rg += hq_rg(rgba_next);
    bc += hq_bc(rgba_next);
  }
  atomicAdd(accum + 2 * (uint64_t)pix, rg);
  atomicAdd(accum + 2 * (uint64_t)pix + 1, bc);
}

__device__ __noinline__ void hq_deferred(const CertParams& P, const long long* sF, uint4 p,
                                         const unsigned long long* keys, unsigned long long* accum, uint32_t eps_num,
                                         uint32_t eps_den) {
  const CertFrag f = classify_cert(P, sF, p);
  bool accept;
  uint32_t pix = f.pixel;
  if (hq_decide(P, f, keys, eps_num, eps_den, &accept)) {
    unsigned long long q;
    accept = project_fp64(P.v, __uint_as_float(p.x), __uint_as_float(p.y), __uint_as_float(p.z), &pix, &q) &&
             in_band(q, keys[pix] >> 24, P.v.nq, eps_num, eps_den);
  }
  if (accept) hq_add(accum, pix, p.w);
}

// Per-pixel accept bounds of the HQ band (Section 2.2) for one pass 2: bounds[i] = {qmin, qmin + floor(eps_num
// (qmin + Nq) / eps_den)} with qmin the pixel's stored code. A code q passes in_band against qmin iff
// bounds.x <= q <= bounds.y whenever eps_num (2^40 + Nq) + eps_den 2^40 <= 2^64 (band_bounds_exact): then
// eps_den (q - qmin) cannot wrap into the band for q < qmin, and qmin + floor(...) cannot wrap either. One thread
// per pixel: 8 bytes read, 16 written. The division by eps_den is a multiplication by its invariant-divisor
// magic number (DivMagic).
struct DivMagic {
  unsigned long long m;
  uint32_t sh1, sh2;
};

// Exact unsigned 64-bit division by an invariant d >= 1 (Granlund and Montgomery, "Division by invariant integers
// using multiplication", 1994, unsigned case with N = 64): with l = ceil(log2 d), m = floor(2^64 (2^l - d) / d)
// + 1 < 2^64, t = floor(m n / 2^64): floor(n / d) = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0) for every
// 0 <= n < 2^64.
inline DivMagic div_magic(uint32_t d) {
  uint32_t l = 0;
  while (l < 32 && (1ull << l) < d) ++l;
  DivMagic r;
  r.m = (unsigned long long)((((unsigned __int128)((1ull << l) - d)) << 64) / d) + 1ull;
  r.sh1 = l < 1 ? l : 1;
  r.sh2 = l > 1 ? l - 1 : 0;
  return r;
}

__device__ __forceinline__ unsigned long long div_by(unsigned long long n, const DivMagic& D) {
  const unsigned long long t = __umul64hi(D.m, n);
  return (t + ((n - t) >> D.sh1)) >> D.sh2;
}

__global__ void k_band_bounds(const unsigned long long* __restrict__ keys, uint64_t npx, unsigned long long nq,
                              uint32_t eps_num, DivMagic D, ulonglong2* __restrict__ bounds) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < npx; i += (uint64_t)gridDim.x * blockDim.x) {
    const unsigned long long qmin = keys[i] >> 24;
    bounds[i] = make_ulonglong2(qmin, qmin + div_by((unsigned long long)eps_num * (qmin + nq), D));
  }
}

inline bool band_bounds_exact(unsigned long long nq, uint32_t eps_num, uint32_t eps_den) {
  const unsigned __int128 lhs = (unsigned __int128)eps_num * (((unsigned __int128)1 << 40) + nq) +
                                ((unsigned __int128)eps_den << 40);
  return lhs <= ((unsigned __int128)1 << 64);
}

// A decided code against the band: through the pixel's bounds when they are given, else in_band on its stored key.
__device__ __forceinline__ bool band_accept(const ulonglong2* bounds, const unsigned long long* keys, uint32_t pix,
                                            unsigned long long q, unsigned long long nq, uint32_t eps_num,
                                            uint32_t eps_den) {
  if (bounds) {
    const ulonglong2 b = __ldcg(bounds + pix);
    return q >= b.x && q <= b.y;
  }
  return in_band(q, stored_key(keys, pix) >> 24, nq, eps_num, eps_den);
}

// Pass 2 (Section 2.2) with the certified transform, same two tiers and the same point staging as pass 1, at
// 64 registers and 4 blocks per SM with both points of a lane classified before their stored-key reads (the
// fastest measured shape: 1.5 % faster than one point at a time at 48 registers and 5 blocks).
#ifndef PCR_HQ_MIN_BLOCKS
#define PCR_HQ_MIN_BLOCKS 4
#endif
// kBand: only the points whose bit is set in band_mask (written by pass 1 for the same points and view, see
// BandMask) can be accepted; each warp appends them to a shared-memory candidate queue and classifies them 32
// at a time, so the cost follows the points that may be in the band.
// bounds (exact transform): the pixels' accept bounds from k_band_bounds for this eps, or null (in_band on the
// stored key). Tier 2 and the arbiter always test against the stored key.
template <bool kApprox, bool kMerge, bool kRing, bool kBand = false>
__global__ void __launch_bounds__(kCertThreads, PCR_HQ_MIN_BLOCKS) k_hq_cert(
    const uint4* __restrict__ pts, uint64_t n, const __grid_constant__ CertParams P,
    const unsigned long long* __restrict__ keys, unsigned long long* __restrict__ accum, uint32_t eps_num,
    uint32_t eps_den, uint32_t* __restrict__ status, const long long* __restrict__ table,
    const uint32_t* __restrict__ band_mask = nullptr, const ulonglong2* __restrict__ bounds = nullptr) {
  __shared__ long long sF[3 * kTableEntries];
  __shared__ uint4 queue[kCertWarps][kQueue];
  __shared__ uint4 cand_queue[kBand ? kCertWarps : 1][kQueue];
  __shared__ __align__(128) uint4 ring[kCertWarps][2][kTile];
  __shared__ __align__(8) uint64_t bars[kCertWarps][2];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  if (kRing && lane == 0) ring_init(bars[warp]);
  __syncwarp();
  if (!kApprox) load_table(P, table, sF);
  uint4* q = queue[warp];
  uint32_t qn = 0;
  // The additions of accepted fragments: warp-level same-pixel merging (kMerge), else lane pairs.
  auto add = [&](bool accept, uint32_t pix, uint32_t rgba) {
    if constexpr (kMerge)
      commit_add<true>(accept, pix, rgba, accum, lane);
    else
      commit_add_pairs(accept, pix, rgba, accum, lane);
  };
  // Double-float mode, per point: the evaluation, the band test against the stored key, the additions.
  auto point_df = [&](const uint4& p, bool valid) {
    bool accept = false;
    uint32_t pix = 0;
    if (valid) {
      const CertFrag f = classify_df(P, p);
      pix = f.pixel;
      hq_decide(P, f, keys, eps_num, eps_den, &accept);
    }
    add(accept, pix, p.w);
  };
  // Exact mode, tier 1 of one point: decided (exact code), or deferred to tier 2 (undecided pixel, or a code
  // undecided between two neighbours: rare, and settling it here would cost every point a second band test).
  auto frag = [&](const uint4& p, bool valid, bool& exact, bool& defer, uint32_t& pix, unsigned long long& qc) {
    exact = false;
    defer = false;
    pix = 0;
    qc = 0;
    if (valid) {
      const FastFrag f = classify_fast(P, sF, p);
      pix = f.pixel;
      exact = f.state == kExact;
      defer = f.state >= kAmbiguous;
      qc = code_from_fixed(f.a1, f.a2);
    }
  };
  // kBand: one candidate per lane; the point's band test and additions, or its deferral.
  uint4* cq = cand_queue[kBand ? warp : 0];
  uint32_t cn = 0;
  auto candidate = [&](const uint4& p, bool valid) {
    bool e, d;
    uint32_t x;
    unsigned long long qc;
    frag(p, valid, e, d, x, qc);
    add(e && band_accept(bounds, keys, x, qc, P.v.nq, eps_num, eps_den), x, p.w);
    defer_points(d, p, q, qn, lane, [&](const uint4& dd) { hq_deferred(P, sF, dd, keys, accum, eps_num, eps_den); });
  };
  // Both points of the lane's tile are classified first, so that their two stored-key reads are in flight
  // together; then the band tests, the additions, the deferrals.
  const bool done = stream_tiles<kRing>(pts, n, ring[warp], bars[warp], lane,
                                        [&](const uint4& p0, bool v0, const uint4& p1, bool v1, uint64_t tile) {
    if constexpr (kBand) {
      // the tile's two words (the same in every lane); each half's set points are appended to the queue, which
      // is drained 32 at a time (at most 31 + 32 entries: the queue holds 64)
      const uint2 bits = reinterpret_cast<const uint2*>(band_mask)[tile];
      const uint32_t below = (1u << lane) - 1u;
      auto push = [&](uint32_t word, const uint4& p) {
        if ((word >> lane) & 1u) cq[cn + __popc(word & below)] = p;
        cn += __popc(word);
        __syncwarp();
        if (cn >= 32u) {
          cn -= 32u;
          const uint4 c = cq[cn + lane];
          __syncwarp();
          candidate(c, true);
        }
      };
      push(bits.x, p0);
      push(bits.y, p1);
      (void)v0;
      (void)v1;
    } else if constexpr (kApprox) {
      point_df(p0, v0);
      point_df(p1, v1);
    } else {
      bool e0, e1, d0, d1;
      uint32_t x0, x1;
      unsigned long long q0, q1;
      frag(p0, v0, e0, d0, x0, q0);
      frag(p1, v1, e1, d1, x1, q1);
      bool a0, a1;
      if (bounds) {
        const ulonglong2 b0 = e0 ? __ldcg(bounds + x0) : make_ulonglong2(1ull, 0ull);
        const ulonglong2 b1 = e1 ? __ldcg(bounds + x1) : make_ulonglong2(1ull, 0ull);
        a0 = q0 >= b0.x && q0 <= b0.y;
        a1 = q1 >= b1.x && q1 <= b1.y;
      } else {
        const unsigned long long m0 = e0 ? stored_key(keys, x0) >> 24 : 0ull;
        const unsigned long long m1 = e1 ? stored_key(keys, x1) >> 24 : 0ull;
        a0 = e0 && in_band(q0, m0, P.v.nq, eps_num, eps_den);
        a1 = e1 && in_band(q1, m1, P.v.nq, eps_num, eps_den);
      }
      add(a0, x0, p0.w);
      add(a1, x1, p1.w);
      auto tier2 = [&](const uint4& d) { hq_deferred(P, sF, d, keys, accum, eps_num, eps_den); };
      defer_points(d0, p0, q, qn, lane, tier2);
      defer_points(d1, p1, q, qn, lane, tier2);
    }
  });
  if (!done && lane == 0) atomicOr(status, kStatusTimeout);
  if constexpr (kBand) {  // the last candidates (fewer than 32)
    const uint4 c = cq[lane < cn ? lane : 0];
    __syncwarp();
    candidate(c, lane < cn);
  }
  if (!kApprox && lane < qn) hq_deferred(P, sF, q[lane], keys, accum, eps_num, eps_den);
}

// ---------------------------------------------------------------------------------------------- launch

// Launch tuning (per framebuffer, see pcr_set_tuning): same-pixel merging within a warp, grid size, point
// staging (0: direct loads, 1: bulk-copy rings).
struct Tuning {
  int merge = 0;
  int blocks_per_sm = 8;
  int staging = 0;
  int band_filter = 0;  // pass 1 writes the band mask for eps <= band_num / band_den (see BandMask)
  uint32_t band_num = 1, band_den = 100;
  int band_bounds = 0;  // pass 2 tests decided codes against per-pixel bounds (k_band_bounds)
};

inline unsigned cert_grid(uint64_t n, int sms, int per_sm) {
  const uint64_t need = (n + kCertThreads - 1) / kCertThreads, cap = (uint64_t)sms * per_sm;
  return (unsigned)(need < cap ? need : cap);
}

// Resident blocks per SM of a kernel (cached per process; every device here is the same GB300 part).
template <typename K>
inline int resident_blocks(K kernel) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kCertThreads, 0) != cudaSuccess || b < 1) {
    cudaGetLastError();
    b = 1;
  }
  return b;
}

// Grid of a persistent grid-stride launch: never more blocks than can be resident at once.
inline unsigned persistent_grid(int resident, uint64_t n, int sms, int per_sm) {
  return cert_grid(n, sms, per_sm < resident ? per_sm : resident);
}

// table: device copy of P.F (or null: the kernels read it from the parameter block); for PIECEWISE views
// (P.n_pw > 0) the device copy of all the ranges' tables, required.
template <bool kApprox, bool kMerge, bool kStats, bool kRing, int kPw, bool kBand = false>
inline void raster_launch5(const uint4* pts, uint64_t n, const CertParams& P, unsigned long long* keys,
                           unsigned long long* stats, uint32_t* status, int sms, int per_sm, cudaStream_t s,
                           const long long* table, BandMask band = BandMask{nullptr, 1u, 0u, 0ull}) {
  auto kernel = k_raster_cert<kApprox, kMerge, kStats, kRing, kPw, kBand>;
  if constexpr (kPw) {
    // the ranges' tables in dynamic shared memory: up to kMaxRanges * 12 KB (opt in above 48 KB once)
    static const bool opted = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)(kMaxRanges * sizeof(P.F))) == cudaSuccess;
    (void)opted;
    const size_t dyn = (size_t)P.n_pw * sizeof(P.F);
    int resident = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, kernel, kCertThreads, dyn) != cudaSuccess ||
        resident < 1) {
      cudaGetLastError();
      resident = 1;
    }
    kernel<<<persistent_grid(resident, n, sms, per_sm), kCertThreads, dyn, s>>>(pts, n, P, keys, stats, status, table,
                                                                               band);
  } else {
    static const int resident = resident_blocks(kernel);  // per instantiation
    kernel<<<persistent_grid(resident, n, sms, per_sm), kCertThreads, 0, s>>>(pts, n, P, keys, stats, status, table,
                                                                             band);
  }
}

template <bool kApprox, bool kMerge, bool kStats, bool kRing>
inline void raster_launch4(const uint4* pts, uint64_t n, const CertParams& P, unsigned long long* keys,
                           unsigned long long* stats, uint32_t* status, int sms, int per_sm, cudaStream_t s,
                           const long long* table, BandMask band = BandMask{nullptr, 1u, 0u, 0ull}) {
  if constexpr (!kApprox && !kStats) {
    if (band.mask && P.n_pw == 0) {  // also write the band mask for pass 2
      raster_launch5<false, kMerge, false, kRing, 0, true>(pts, n, P, keys, nullptr, status, sms, per_sm, s, table,
                                                           band);
      return;
    }
  }
  if (!kApprox && P.n_pw > 2)
    raster_launch5<false, kMerge, kStats, kRing, 2>(pts, n, P, keys, stats, status, sms, per_sm, s, table);
  else if (!kApprox && P.n_pw > 0)
    raster_launch5<false, kMerge, kStats, kRing, 1>(pts, n, P, keys, stats, status, sms, per_sm, s, table);
  else
    raster_launch5<kApprox, kMerge, kStats, kRing, 0>(pts, n, P, keys, stats, status, sms, per_sm, s, table);
}

// Pass 1 with the tuning's staging; the tier counters (stats) only with the exact transform, no merging.
template <bool kApprox, bool kMerge>
inline void raster_launch(const uint4* pts, uint64_t n, const CertParams& P, unsigned long long* keys,
                          unsigned long long* stats, uint32_t* status, int sms, int per_sm, cudaStream_t s,
                          const long long* table = nullptr, int staging = 0,
                          BandMask band = BandMask{nullptr, 1u, 0u, 0ull}) {
  if (stats && !kApprox && !kMerge)
    staging ? raster_launch4<false, false, true, true>(pts, n, P, keys, stats, status, sms, per_sm, s, table)
            : raster_launch4<false, false, true, false>(pts, n, P, keys, stats, status, sms, per_sm, s, table);
  else
    staging ? raster_launch4<kApprox, kMerge, false, true>(pts, n, P, keys, nullptr, status, sms, per_sm, s, table,
                                                           band)
            : raster_launch4<kApprox, kMerge, false, false>(pts, n, P, keys, nullptr, status, sms, per_sm, s, table,
                                                            band);
}

// The certified constants of a view, prepared on this thread and kept for the next call with the same view
// and mode (prepare_cert builds a 12 KB exact table: ~14 us of host time per call). Returns false when the
// view is outside the single-precision preconditions.
// tables (optional): the view's depth tables, block r for PIECEWISE range r (P->n_pw blocks; one for LINEAR
// and METRIC), to be copied to the device.
inline bool cached_cert(const DevView& v, bool approximate, const CertParams** out,
                        const long long** tables = nullptr) {
  static thread_local CertParams P;
  static thread_local long long T[kMaxRanges][3][kTableEntries];
  static thread_local DevView last_v;
  static thread_local int last = -1;  // -1: nothing cached; else approximate (0/1) of the cached view
  static thread_local bool last_ok = false;
  if (last != (approximate ? 1 : 0) || std::memcmp(&last_v, &v, sizeof(DevView)) != 0) {
    last_ok = host::prepare_cert(v, approximate, &P, T);
    std::memcpy(&last_v, &v, sizeof(DevView));
    last = approximate ? 1 : 0;
  }
  *out = &P;
  if (tables) *tables = &T[0][0][0];
  return last_ok;
}

// Blocks of the depth tables of prepared constants (the device copy's size in tables of 3 * kTableEntries).
inline int table_blocks(const CertParams& P) { return P.n_pw > 0 ? P.n_pw : 1; }

// Pass 1 for a view with n >= 1 points. status: the framebuffer's status word (timeout bit).
// band (mask non-null): also write the band mask for pass 2 (used only with the exact transform on LINEAR or
// METRIC views; the caller checks that before relying on it).
inline bool launch_raster_certified(const uint4* pts, uint64_t n, const DevView& v, bool approximate,
                                    unsigned long long* keys, uint32_t* status, int sms, cudaStream_t s,
                                    unsigned long long* stats = nullptr, const Tuning& t = Tuning(),
                                    const long long* table = nullptr, BandMask band = BandMask{nullptr, 1u, 0u, 0ull}) {
  const CertParams* Pp = nullptr;
  const unsigned grid = cert_grid(n, sms, t.blocks_per_sm);
  // PIECEWISE views need the device copy of their tables
  if (!cached_cert(v, approximate, &Pp) || (Pp->n_pw > 0 && table == nullptr)) {
    k_raster_fp64<<<grid, 256, 0, s>>>(pts, n, v, keys);
    return true;
  }
  const int b = t.blocks_per_sm, g = t.staging;
  if (approximate)
    t.merge ? raster_launch<true, true>(pts, n, *Pp, keys, stats, status, sms, b, s, table, g)
            : raster_launch<true, false>(pts, n, *Pp, keys, stats, status, sms, b, s, table, g);
  else
    t.merge ? raster_launch<false, true>(pts, n, *Pp, keys, stats, status, sms, b, s, table, g, band)
            : raster_launch<false, false>(pts, n, *Pp, keys, stats, status, sms, b, s, table, g, band);
  return true;
}

template <bool kApprox, bool kMerge, bool kRing, bool kBand = false>
inline void hq_launch4(const uint4* pts, uint64_t n, const CertParams& P, const unsigned long long* keys,
                       unsigned long long* accum, uint32_t eps_num, uint32_t eps_den, uint32_t* status, int sms,
                       int per_sm, cudaStream_t s, const long long* table, const uint32_t* band_mask,
                       const ulonglong2* bounds) {
  static const int resident = resident_blocks(k_hq_cert<kApprox, kMerge, kRing, kBand>);  // one per instantiation
  const unsigned grid = persistent_grid(resident, n, sms, per_sm);
  k_hq_cert<kApprox, kMerge, kRing, kBand><<<grid, kCertThreads, 0, s>>>(pts, n, P, keys, accum, eps_num, eps_den,
                                                                         status, table, band_mask, bounds);
}

// band_mask (exact transform only): pass 1's band mask of the same points and view, or null. bounds (exact
// transform only): the pixels' accept bounds for this eps (k_band_bounds), or null.
template <bool kApprox, bool kMerge>
inline void hq_launch(const uint4* pts, uint64_t n, const CertParams& P, const unsigned long long* keys,
                      unsigned long long* accum, uint32_t eps_num, uint32_t eps_den, uint32_t* status, int sms,
                      int per_sm, cudaStream_t s, const long long* table = nullptr, int staging = 0,
                      const uint32_t* band_mask = nullptr, const ulonglong2* bounds = nullptr) {
  if constexpr (!kApprox) {
    if (band_mask) {
      staging ? hq_launch4<false, kMerge, true, true>(pts, n, P, keys, accum, eps_num, eps_den, status, sms, per_sm, s,
                                                      table, band_mask, bounds)
              : hq_launch4<false, kMerge, false, true>(pts, n, P, keys, accum, eps_num, eps_den, status, sms, per_sm,
                                                       s, table, band_mask, bounds);
      return;
    }
  } else {
    bounds = nullptr;
  }
  staging ? hq_launch4<kApprox, kMerge, true>(pts, n, P, keys, accum, eps_num, eps_den, status, sms, per_sm, s, table,
                                              nullptr, bounds)
          : hq_launch4<kApprox, kMerge, false>(pts, n, P, keys, accum, eps_num, eps_den, status, sms, per_sm, s, table,
                                               nullptr, bounds);
}

// Pass 2 for a view with n >= 1 points. status: the framebuffer's status word (timeout bit). band_mask: see
// hq_launch. bounds_buf: room for the accept bounds of every pixel (npx entries), or null; with the exact
// transform and band_bounds_exact they are computed (k_band_bounds) and pass 2 tests against them. Returns the
// number of kernels launched.
inline int launch_hq_certified(const uint4* pts, uint64_t n, const DevView& v, bool approximate,
                               const unsigned long long* keys, unsigned long long* accum, uint32_t eps_num,
                               uint32_t eps_den, uint32_t* status, int sms, cudaStream_t s,
                               const Tuning& t = Tuning(), const long long* table = nullptr,
                               const uint32_t* band_mask = nullptr, ulonglong2* bounds_buf = nullptr) {
  const CertParams* Pp = nullptr;
  const unsigned grid = cert_grid(n, sms, t.blocks_per_sm);
  if (!cached_cert(v, approximate, &Pp) || Pp->n_pw > 0) {  // (HQ takes LINEAR or METRIC views only)
    k_hq_fp64<<<grid, 256, 0, s>>>(pts, n, v, keys, accum, eps_num, eps_den);
    return 1;
  }
  const int b = t.blocks_per_sm, g = t.staging;
  if (approximate) {
    t.merge ? hq_launch<true, true>(pts, n, *Pp, keys, accum, eps_num, eps_den, status, sms, b, s, table, g)
            : hq_launch<true, false>(pts, n, *Pp, keys, accum, eps_num, eps_den, status, sms, b, s, table, g);
    return 1;
  }
  const ulonglong2* bounds = nullptr;
  if (bounds_buf && band_bounds_exact(v.nq, eps_num, eps_den)) {
    const uint64_t npx = (uint64_t)v.width * v.height;
    const unsigned bgrid = (unsigned)((npx + 255) / 256 < (uint64_t)sms * 8 ? (npx + 255) / 256 : (uint64_t)sms * 8);
    k_band_bounds<<<bgrid, 256, 0, s>>>(keys, npx, v.nq, eps_num, div_magic(eps_den), bounds_buf);
    bounds = bounds_buf;
  }
  t.merge ? hq_launch<false, true>(pts, n, *Pp, keys, accum, eps_num, eps_den, status, sms, b, s, table, g,
                                   band_mask, bounds)
          : hq_launch<false, false>(pts, n, *Pp, keys, accum, eps_num, eps_den, status, sms, b, s, table, g,
                                    band_mask, bounds);
  return bounds ? 2 : 1;
}

}  // namespace pcr
