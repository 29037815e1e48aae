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
// A point whose depth code is undecided between two neighbours is sent on only when it could still win
// its pixel (its smaller candidate key is below the key the framebuffer holds); a point whose cull or
// pixel is undecided, and those, go through the FP64 definition directly (the arbiter). The output is
// therefore bit-identical to the FP64 definition.
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
  DevView v;                          // the FP64 definition (for the arbiter)
  long long F[3][kTableEntries];      // t-row fixed-point coefficients, index (sign << 8) | exponent
  float H[3][4], L[3][4];             // double-float splits of the rows clip x, clip y, w
  float kappa;                        // double-float error bound factor (relative to T)
  float t_c1, t_c2;                   // FP64-rounding + fixed-point bound of t: t_c1 * T_t + t_c2
  float Af[3], Bf;                    // float approximations of A_j and B (for T_t)
  uint32_t B0, B1, B2;                // B * 2^40 as a 96-bit two's-complement integer (low word first)
  int32_t e_max[3];                   // largest biased exponent of x, y, z with a usable table entry
  long long qn_safe, qn_cull, qf_safe, qf_cull;  // depth-cull thresholds in code space
  // approximate (double-float, no arbiter) mode
  float near_h, near_l, far_h, far_l, S_h, S_l;
  int32_t approximate;
  int32_t linear;
};

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

// Fills P for the view; false when the view is outside the certified evaluation's preconditions (the
// caller then uses the FP64 kernels, which accept every valid view).
inline bool prepare_cert(const DevView& v, bool approximate, CertParams* P) {
  std::memset(P, 0, sizeof(*P));
  P->v = v;
  P->approximate = approximate ? 1 : 0;
  if (v.depth_mode != 0 && v.depth_mode != 1) return false;  // piecewise: FP64 kernels
  P->linear = v.depth_mode == 0;
  if (!(v.near_ >= 0x1p-60) || !(v.far_ < 0x1p100)) return false;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 4; ++c)
      if (!split_float(v.m[4 * r + c], &P->H[r][c], &P->L[r][c])) return false;
  P->kappa = 40.0f * 0x1p-48f * (1.0f + 0x1p-20f);
  const double S = v.scale;
  if (!(S > 0.0) || !(S < 0x1p100)) return false;
  two_float(v.near_, &P->near_h, &P->near_l);
  two_float(v.far_, &P->far_h, &P->far_l);
  two_float(S, &P->S_h, &P->S_l);
  // t = sum_j A_j X_j + B, A_j = S * M[3][j], B = S * (M[3][3] - near) (LINEAR) or S * M[3][3] (METRIC)
  const double* m3 = v.m + 8;
  for (int j = 0; j < 3; ++j) {
    const double a = S * m3[j];
    if (!(std::fabs(a) < 0x1p80)) return false;  // keeps the subnormal shortcut's error below 2^-46
    P->Af[j] = (float)a;
    P->e_max[j] = 254;
    for (int e = 0; e < kTableExp; ++e) {
      const int ee = e == 0 ? 1 : e;  // subnormals share exponent 1's scale (see the device loop)
      __int128 f;
      const bool ok = e < 255 && fixed_mul(S, m3[j], ee - 150 + kFixedFracBits, &f) &&
                      f < ((__int128)1 << 62) && f > -((__int128)1 << 62);
      if (!ok) {
        if (P->e_max[j] >= e) P->e_max[j] = e - 1;
        f = 0;
      }
      P->F[j][e] = (long long)f;
      P->F[j][kTableExp + e] = -(long long)f;
    }
    if (P->e_max[j] < 127) return false;  // coordinates of magnitude 1 would not be usable
  }
  __int128 b, bn = 0;
  if (!fixed_mul(S, m3[3], kFixedFracBits, &b)) return false;
  if (P->linear && !fixed_mul(S, v.near_, kFixedFracBits, &bn)) return false;
  b -= bn;
  if (b >= ((__int128)1 << 94) || b <= -((__int128)1 << 94)) return false;
  const unsigned __int128 bu = (unsigned __int128)b;
  P->B0 = (uint32_t)bu;
  P->B1 = (uint32_t)(bu >> 32);
  P->B2 = (uint32_t)(bu >> 64);
  const double bd = S * m3[3] - (P->linear ? S * v.near_ : 0.0);
  if (!(std::fabs(bd) < 1e38)) return false;
  P->Bf = (float)bd;
  // |t_FP64 - t| <= u64 * (5.2 * T_t + 3.1 * S * near) (LINEAR; the near term is absent for METRIC);
  // the fixed-point sum adds < 2^-15; 2^-13 covers both that and the float evaluation of the bound.
  const double u64 = 0x1p-53;
  P->t_c1 = (float)(5.2 * u64 * (1.0 + 0x1p-18));
  P->t_c2 = (float)((P->linear ? 3.1 * u64 * S * v.near_ : 0.0) + 0x1p-13);
  // depth-cull thresholds: T_n, T_f are the FP64 codes of the near and far planes (monotone rounding:
  // t > T_n => w >= near, t < T_n => w < near, t < T_f => w < far, t > T_f => w >= far)
  const double Tn = P->linear ? 0.0 : v.near_ * S;
  const double Tf = P->linear ? (v.far_ - v.near_) * S : v.far_ * S;
  if (!(Tf < 0x1p62)) return false;
  P->qn_safe = (long long)std::floor(Tn) + 1;
  P->qn_cull = (long long)std::floor(Tn) - 1;
  P->qf_safe = (long long)std::floor(Tf) - 1;
  P->qf_cull = (long long)std::floor(Tf) + 1;
  return true;
}

}  // namespace host

// ---------------------------------------------------------------------------------------------- device

enum : uint32_t { kCulled = 0, kExact = 1, kAmbiguous = 2, kHard = 3 };

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

// Classifies one point. F points at the block's shared-memory copy of P.F.
__device__ __forceinline__ CertFrag classify_cert(const CertParams& P, const long long* __restrict__ F, uint4 p) {
  CertFrag out{kCulled, 0u, 0};
  const uint32_t bx = p.x, by = p.y, bz = p.z;
  const uint32_t ex = (bx >> 23) & 0xFFu, ey = (by >> 23) & 0xFFu, ez = (bz >> 23) & 0xFFu;
  // any NaN or infinite coordinate makes w NaN or infinite in FP64: culled
  if (ex == 0xFFu || ey == 0xFFu || ez == 0xFFu) return out;
  if ((int)ex > P.e_max[0] || (int)ey > P.e_max[1] || (int)ez > P.e_max[2]) {
    out.state = kHard;
    return out;
  }
  // ---- depth code: t * 2^40 as a 96-bit integer
  uint32_t a0 = P.B0, a1 = P.B1, a2 = P.B2;
  // a subnormal coordinate takes the implicit bit too; its table entry uses exponent 1's scale, so the
  // product is A * (X + 2^-126 sign(X)): an error below |A| 2^-126, far inside the bound
  mac96((bx & 0x7FFFFFu) | 0x800000u, F[(bx >> 23)], a0, a1, a2);
  mac96((by & 0x7FFFFFu) | 0x800000u, F[kTableEntries + (by >> 23)], a0, a1, a2);
  mac96((bz & 0x7FFFFFu) | 0x800000u, F[2 * kTableEntries + (bz >> 23)], a0, a1, a2);
  const float x = __uint_as_float(bx), y = __uint_as_float(by), z = __uint_as_float(bz);
  const long long qc = (long long)(int32_t)a2 * 16777216LL + (long long)(a1 >> 8);  // floor(t)
  const float frac = __fsub_rn(__uint_as_float(0x3F800000u | (__funnelshift_r(a0, a1, 8) >> 9)), 1.0f);
  const float Tt = __fadd_rn(__fadd_rn(__fadd_rn(fabsf(__fmul_rn(P.Af[0], x)), fabsf(__fmul_rn(P.Af[1], y))),
                                       fabsf(__fmul_rn(P.Af[2], z))), fabsf(P.Bf));
  const float D = __fadd_rn(__fmaf_rn(P.t_c1, Tt, P.t_c2), 0x1p-22f);
  long long qa, qb;
  bool exact;
  if (D >= 0.5f) {
    out.state = kHard;
    return out;
  }
  if (frac > D && frac < __fsub_rn(1.0f, D)) {
    qa = qb = qc;
    exact = true;
  } else {
    qa = frac < 0.5f ? qc - 1 : qc;
    qb = qa + 1;
    exact = false;
  }
  if (qb <= P.qn_cull || qa >= P.qf_cull) return out;  // culled by the clip planes
  if (qa < P.qn_safe || qb > P.qf_safe) {
    out.state = kHard;
    return out;
  }
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
  if (!(fx >= 0.0f && fx < P.v.fwidth && fy >= 0.0f && fy < P.v.fheight)) return out;
  out.pixel = (uint32_t)__float2int_rz(fy) * (uint32_t)P.v.width + (uint32_t)__float2int_rz(fx);
  const long long qmax = (long long)kQMax;
  if (qa >= qmax) exact = true;  // both candidates cap to 2^40 - 2
  out.q = qa < qmax ? qa : qmax;
  out.state = exact ? kExact : kAmbiguous;
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

// Pass 1 (Section 2.1) with the certified transform. Undecided depth codes are resolved by occlusion
// when possible; everything else undecided goes through the FP64 definition.
template <bool kApprox>
__global__ void __launch_bounds__(256) k_raster_cert(const uint4* __restrict__ pts, uint64_t n,
                                                     const __grid_constant__ CertParams P,
                                                     unsigned long long* __restrict__ keys,
                                                     unsigned long long* __restrict__ stats) {
  __shared__ long long sF[3 * kTableEntries];
  if (!kApprox) load_table(P, sF);
  unsigned c_exact = 0, c_amb = 0, c_amb_fp64 = 0, c_hard = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint4 p = ld_stream16(pts + i);
    const CertFrag f = kApprox ? classify_df(P, p) : classify_cert(P, sF, p);
    if (f.state == kExact) {
      ++c_exact;
      atomicMin(keys + f.pixel, make_key((unsigned long long)f.q, p.w));
      continue;
    }
    bool arbiter = f.state == kHard;
    if (f.state == kAmbiguous) {
      ++c_amb;
      // the smaller candidate cannot win when it is not below the stored key (keys only decrease)
      arbiter = make_key((unsigned long long)f.q, p.w) < keys[f.pixel];
      c_amb_fp64 += arbiter;
    } else {
      c_hard += arbiter;
    }
    if (arbiter) {
      uint32_t pix;
      unsigned long long q;
      if (project_fp64(P.v, __uint_as_float(p.x), __uint_as_float(p.y), __uint_as_float(p.z), &pix, &q))
        atomicMin(keys + pix, make_key(q, p.w));
    }
  }
  if (stats) {
    atomicAdd(stats + 0, (unsigned long long)c_exact);
    atomicAdd(stats + 1, (unsigned long long)c_amb);
    atomicAdd(stats + 2, (unsigned long long)c_amb_fp64);
    atomicAdd(stats + 3, (unsigned long long)c_hard);
  }
}

// Pass 2 (Section 2.2) with the certified transform.
template <bool kApprox>
__global__ void __launch_bounds__(256) k_hq_cert(const uint4* __restrict__ pts, uint64_t n,
                                                 const __grid_constant__ CertParams P,
                                                 const unsigned long long* __restrict__ keys,
                                                 unsigned long long* __restrict__ accum, uint32_t eps_num,
                                                 uint32_t eps_den) {
  __shared__ long long sF[3 * kTableEntries];
  if (!kApprox) load_table(P, sF);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint4 p = ld_stream16(pts + i);
    const CertFrag f = kApprox ? classify_df(P, p) : classify_cert(P, sF, p);
    if (f.state == kCulled) continue;
    uint32_t pix = f.pixel;
    unsigned long long q = (unsigned long long)f.q;
    bool accept = false;
    bool arbiter = f.state == kHard;
    if (!arbiter) {
      const unsigned long long qmin = keys[pix] >> 24;
      accept = in_band(q, qmin, P.v.nq, eps_num, eps_den);
      if (f.state == kAmbiguous) {
        const unsigned long long q2 = q + 1 < kQMax ? q + 1 : kQMax;
        arbiter = accept != in_band(q2, qmin, P.v.nq, eps_num, eps_den);
      }
    }
    if (arbiter) {
      accept = false;
      if (project_fp64(P.v, __uint_as_float(p.x), __uint_as_float(p.y), __uint_as_float(p.z), &pix, &q))
        accept = in_band(q, keys[pix] >> 24, P.v.nq, eps_num, eps_den);
    }
    if (accept) {
      atomicAdd(accum + 2 * (uint64_t)pix, hq_rg(p.w));
      atomicAdd(accum + 2 * (uint64_t)pix + 1, hq_bc(p.w));
    }
  }
}

// ---------------------------------------------------------------------------------------------- launch

inline unsigned cert_grid(uint64_t n, int sms) {
  const uint64_t need = (n + 255) / 256, cap = (uint64_t)sms * 8;
  return (unsigned)(need < cap ? need : cap);
}

inline bool launch_raster_certified(const uint4* pts, uint64_t n, const DevView& v, bool approximate,
                                    unsigned long long* keys, int sms, cudaStream_t s,
                                    unsigned long long* stats = nullptr) {
  static thread_local CertParams P;  // 12.8 KB: kept off the stack
  if (!host::prepare_cert(v, approximate, &P)) {
    k_raster_fp64<<<cert_grid(n, sms), 256, 0, s>>>(pts, n, v, keys);
    return true;
  }
  if (approximate)
    k_raster_cert<true><<<cert_grid(n, sms), 256, 0, s>>>(pts, n, P, keys, stats);
  else
    k_raster_cert<false><<<cert_grid(n, sms), 256, 0, s>>>(pts, n, P, keys, stats);
  return true;
}

inline bool launch_hq_certified(const uint4* pts, uint64_t n, const DevView& v, bool approximate,
                                const unsigned long long* keys, unsigned long long* accum, uint32_t eps_num,
                                uint32_t eps_den, int sms, cudaStream_t s) {
  static thread_local CertParams P;
  if (!host::prepare_cert(v, approximate, &P)) {
    k_hq_fp64<<<cert_grid(n, sms), 256, 0, s>>>(pts, n, v, keys, accum, eps_num, eps_den);
    return true;
  }
  if (approximate)
    k_hq_cert<true><<<cert_grid(n, sms), 256, 0, s>>>(pts, n, P, keys, accum, eps_num, eps_den);
  else
    k_hq_cert<false><<<cert_grid(n, sms), 256, 0, s>>>(pts, n, P, keys, accum, eps_num, eps_den);
  return true;
}

}  // namespace pcr
