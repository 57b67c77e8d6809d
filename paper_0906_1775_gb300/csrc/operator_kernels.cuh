// Kernels and launch templates of the operator (included once per precision).
//
// Noise weighting N^-1 of Section 5.2 (Eqs. 15-22) fused with the pointing
// gather y = A x (Section 3, Eqs. 3-4) and the scatter A^T w.
//
// Each interval is cut into overlapping windows of M samples whose central
// parts are exact outputs of the banded Toeplitz block (circulant embedding
// with one bandwidth of halo on each side, Section 5.2).  Two real windows
// that use the same filter share one complex FFT of length M (one in the real
// part, one in the imaginary part): the circulant's spectrum is real and even,
// so multiplying by it never mixes the two.  The FFT of length M = N1 * N2 is
// done in four steps (columns, twiddle, rows), with the pointwise filter
// product and the inverse row FFTs in the middle kernel:
//
//   k_f1  gather + N2-point FFTs of the columns n1 (elements n = n1 + N1 n2),
//         twiddle exp(-2 pi i n1 k2 / M), write scratch [k2 position][n1]
//   k_f2  N1-point FFTs of the rows, multiply by the filter spectrum / M,
//         inverse N1-point FFTs, write back
//   k_f3  conjugate twiddle, inverse N2-point FFTs, keep the window's exact
//         outputs and scatter them into the map (or write a timestream)
//
// The row/column FFTs run in shared memory as radix-2 stages fused three at a
// time in registers; forward transforms leave bit-reversed order and the
// inverses consume it, so no reordering pass exists anywhere.
#pragma once

#include <math.h>

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <vector>

#include "internal.cuh"

namespace mm {

namespace {

// Input of the noise weighting: a map (gather y = A x), a float timestream, a
// timestream of the working precision, or the residual timestream d - A x of
// a float timestream d and a map x (the refinement residual b - H x =
// A^T N^-1 (d - A x) in one pass).
enum { IN_MAPX = 0, IN_TODF = 1, IN_TODR = 2, IN_RESX = 3 };
__host__ __device__ constexpr bool gathers(int in) { return in == IN_MAPX || in == IN_RESX; }

// Stokes layouts of the kernels' NS parameter: 1 = T, 3 = IQU on one
// pixelisation, NS_MR = IQU with Q and U on a second pixelisation (Section 6;
// each sample then carries an I pixel and a Q/U pixel of the slot layout).
// NS_OTF_T / NS_OTF_IQU: T / IQU with the pointing expanded on the fly from
// compressed boresight pointing (Section 5.3) instead of read per sample.
// NS_EXT_T / NS_EXT_IQU: T / IQU with extended pointing (Section 6, Eq. 40):
// each sample may add one unit-weight extra column (a row after the sky rows).
constexpr int NS_MR = 4;
constexpr int NS_OTF_T = 5;
constexpr int NS_OTF_IQU = 6;
constexpr int NS_EXT_T = 7;
constexpr int NS_EXT_IQU = 8;
__host__ __device__ constexpr bool polarised(int ns) {
  return ns == 3 || ns == NS_MR || ns == NS_OTF_IQU || ns == NS_EXT_IQU;
}
__host__ __device__ constexpr bool on_the_fly(int ns) { return ns == NS_OTF_T || ns == NS_OTF_IQU; }
__host__ __device__ constexpr bool extended(int ns) { return ns == NS_EXT_T || ns == NS_EXT_IQU; }
// the map layout's gather/scatter of a pointing mode
__host__ __device__ constexpr int map_ns(int ns) {
  return (ns == NS_OTF_T || ns == NS_EXT_T) ? 1 : (ns == NS_OTF_IQU || ns == NS_EXT_IQU) ? 3 : ns;
}
inline int layout(const Plan* p) {
  if (p->otf) return p->n_stokes == 1 ? NS_OTF_T : NS_OTF_IQU;
  if (p->ext) return p->n_stokes == 1 ? NS_EXT_T : NS_EXT_IQU;
  return p->multires ? NS_MR : p->n_stokes;
}
// Calls X(ns) with the compile-time pointing mode ns of `k`.
#define MM_FOR_LAYOUT(k, X)                                                                                  \
  ((k) == 1 ? X(1) : (k) == 3 ? X(3) : (k) == NS_MR ? X(NS_MR) : (k) == NS_OTF_T ? X(NS_OTF_T)             \
   : (k) == NS_OTF_IQU ? X(NS_OTF_IQU) : (k) == NS_EXT_T ? X(NS_EXT_T) : X(NS_EXT_IQU))

struct OpArgs {
  const Tile* tiles;
  int tile0;
  int M, N1, N2, logN1, logN2, B1, logB1, B2;
  const int* pix;
  const float* psi;
  const double2* cs64;
  const float4* csdf;
  const int2* pw;      // (pixel, angle bits) per sample, IQU
  const int* pixq;     // Q/U pixel per sample (multi-resolution plans)
  const int* ext;      // extra column's map row per sample (extended pointing), or NULL
  const int* hwp_base; // first half-wave-plate row of the sample's group (or -1), or NULL
  const float* hwp_ang;
  const float* hwp_tau;
  // compressed pointing (on-the-fly modes)
  const float4* bore;
  const float4* det;
  const int* g2o;
  StepDiv sd;
  int n_per_det, n_det, grid_w, grid_h;
  const void* in;
  long long in_stride;
  const float* in2;      // IN_RESX: the timestream d, in2_stride floats per right-hand side
  long long in2_stride;
  void* out;
  long long out_stride;
  void* scratch;
  const void* H;
  const void* tw;
  int n_rep;          // > 1: map outputs go to replica (blockIdx.x + blockIdx.y) % n_rep, rep_stride apart
  int runs;           // scatter runs of consecutive samples that hit one pixel with one atomic (run_*)
  long long rep_stride;
  const int* skip;    // done flag(s): one shared flag, or one per right-hand side
  int skip_stride;    // 0: *skip covers every tile; > 0: skip[rhs * skip_stride] per lane
};

// A tile is skipped when its solve (or both of its right-hand sides) is done.
__device__ __forceinline__ bool skip_tile(const OpArgs& a, const Tile* T) {
  if (!a.skip) return false;
  if (a.skip_stride == 0) return *a.skip != 0;
  return a.skip[T->l[0].rhs * a.skip_stride] != 0 && a.skip[T->l[1].rhs * a.skip_stride] != 0;
}

// cos 2psi, sin 2psi for the float32 operator.  x = 2 psi (exact) is reduced
// to r = x - 2 pi k, k = rint(x / 2 pi), by Cody and Waite's method (Cody and
// Waite, "Software Manual for the Elementary Functions", 1980): 2 pi is split
// into C1 = 2 pi rounded to float and C2 = 2 pi - C1, and k C1 then k C2 are
// subtracted, each with one fused multiply-add, so the product k C1 is exact
// and r carries at most two roundings (about 2.4e-7 absolute on [-pi, pi]).
// The hardware approximations (absolute error below 4e-7 on [-pi, pi]) take
// it from there: |error| < 1e-6 against the exact weights of the float32
// angle, far inside the float32 operator's own rounding.  The float64
// operator uses correctly rounded float64 weights.
__device__ __forceinline__ void sincos_2psi(float psi, float& s, float& c) {
  const float x = 2.0f * psi;
  const float k = rintf(x * 0.15915494309189535f);
  float r = fmaf(-k, 6.2831854820251465f, x);
  r = fmaf(-k, -1.7484556000744970e-07f, r);
  __sincosf(r, &s, &c);
}
template <typename Real, int NS>
__device__ __forceinline__ Real gather(const Real* x, int p, Real c, Real s);
template <>
__device__ __forceinline__ float gather<float, 1>(const float* x, int p, float, float) {
  return x[p];
}
template <>
__device__ __forceinline__ double gather<double, 1>(const double* x, int p, double, double) {
  return x[p];
}
template <>
__device__ __forceinline__ float gather<float, 3>(const float* x, int p, float c, float s) {
  const float4 m = reinterpret_cast<const float4*>(x)[p];
  return m.x + m.y * c + m.z * s;
}
template <>
__device__ __forceinline__ double gather<double, 3>(const double* x, int p, double c, double s) {
  const double2* xp = reinterpret_cast<const double2*>(x + 4LL * p);
  const double2 u = xp[0], v = xp[1];
  return u.x + u.y * c + v.x * s;
}

// double-float: the map holds float pairs ([n_obs][4] pairs for IQU)
template <>
__device__ __forceinline__ df64 gather<df64, 1>(const df64* x, int p, df64, df64) {
  return x[p];
}
template <>
__device__ __forceinline__ df64 gather<df64, 3>(const df64* x, int p, df64 c, df64 s) {
  const float4* xp = reinterpret_cast<const float4*>(x + 4LL * p);
  const float4 u = xp[0], v = xp[1];
  return df64(u.x, u.y) + df64(u.z, u.w) * c + df64(v.x, v.y) * s;
}

// a kernel's value in its output map's type (double-float results go out as float64)
__device__ __forceinline__ float to_out(float v) { return v; }
__device__ __forceinline__ double to_out(double v) { return v; }
__device__ __forceinline__ double to_out(df64 v) { return to_double(v); }

// Half-wave-plate term of sample n of a lane (rows hb.. hb+31, column 0):
// gather sum_i C_i x_i, or scatter v C_i into each parameter.  Float32
// kernels take the columns in float32, the others in float64.
template <typename Real>
__device__ __noinline__ Real hwp_gather(const Real* x, int hb, int stride, float w, float tau) {
  typedef typename std::conditional<std::is_same<Real, float>::value, float, double>::type W;
  W C[32];
  hwp_columns<W>(w, tau, C);
  W acc = W(0);
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const Real xi = x[(long long)(hb + i) * stride];
    if constexpr (std::is_same<Real, df64>::value) acc += C[i] * to_double(xi);
    else acc += C[i] * (W)xi;
  }
  return Real(acc);
}
// Scatter of one position of a tile lane by a whole (converged) warp: every
// sample of a lane belongs to one interval, so the warp's samples share one
// group; each lane forms its 32 products v C_i, a transposing butterfly of
// 31 shuffles leaves lane i with the warp's sum for parameter i, and each
// lane adds it into the CTA's shared sums `acc` (the group's first row goes
// to *grp); hwp_flush adds those to the map once per CTA.  Lanes without a
// valid sample add zeros.
template <typename Real>
__device__ __noinline__ void hwp_scatter_warp(typename OutT<Real>::type* acc, int* grp, const int* pix, const int* hbp,
                                              const float* ang, const float* tau, int n, bool ok, Real val) {
  typedef typename OutT<Real>::type Out;
  int hb = -1;
  float w = 0.f, t = 0.f;
  if (ok && __ldg(pix + n) >= 0) {
    hb = __ldg(hbp + n);
    if (hb >= 0) {
      w = __ldg(ang + n);
      t = __ldg(tau + n);
    }
  }
  const int g = __reduce_max_sync(0xffffffffu, hb);
  if (g < 0) return;
  const Out v = hb >= 0 ? (Out)to_out(val) : Out(0);
  Out C[32];
  hwp_columns<Out>(w, t, C);
#pragma unroll
  for (int i = 0; i < 32; ++i) C[i] *= v;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 16; k >= 1; k >>= 1) {
    const bool upper = (lane & k) != 0;
#pragma unroll
    for (int i = 0; i < k; ++i) {
      const Out send = upper ? C[i] : C[i + k];
      const Out keep = upper ? C[i + k] : C[i];
      C[i] = keep + __shfl_xor_sync(0xffffffffu, send, k);
    }
  }
  atomicAdd(acc + lane, C[0]);
  if (lane == 0) *grp = g;
}

// The CTA's shared half-wave-plate sums into the map (after a barrier).
template <typename Out>
__device__ __forceinline__ void hwp_flush(Out* y, int stride, const Out* acc, const int* grp, int n_groups) {
  for (int i = threadIdx.x; i < 32 * n_groups; i += blockDim.x) {
    const int g = grp[i / 32];
    if (g >= 0 && acc[i] != Out(0)) atomicAdd(y + (long long)(g + (i & 31)) * stride, acc[i]);
  }
}

// multi-resolution maps: I from slot p, Q and U from slot q
template <typename Real>
__device__ __forceinline__ Real gather_mr(const Real* x, int p, int q, Real c, Real s) {
  if constexpr (std::is_same<Real, float>::value) {
    const float4 m = reinterpret_cast<const float4*>(x)[q];
    return x[4LL * p] + m.y * c + m.z * s;
  } else {
    return x[4LL * p] + x[4LL * q + 1] * c + x[4LL * q + 2] * s;
  }
}

template <typename Real, int NS>
__device__ __forceinline__ void scatter(typename OutT<Real>::type* y, int p, Real v, Real c, Real s);
template <>
__device__ __forceinline__ void scatter<float, 1>(float* y, int p, float v, float, float) {
  atomicAdd(y + p, v);
}
template <>
__device__ __forceinline__ void scatter<double, 1>(double* y, int p, double v, double, double) {
  atomicAdd(y + p, v);
}
template <>
__device__ __forceinline__ void scatter<float, 3>(float* y, int p, float v, float c, float s) {
  atomicAdd(reinterpret_cast<float4*>(y) + p, make_float4(v, v * c, v * s, 0.0f));
}
template <>
__device__ __forceinline__ void scatter<double, 3>(double* y, int p, double v, double c, double s) {
  double* q = y + 4LL * p;
  atomicAdd(q, v);
  atomicAdd(q + 1, v * c);
  atomicAdd(q + 2, v * s);
}
// double-float results are rounded to float64 once per sample and added with
// float64 atomics
template <>
__device__ __forceinline__ void scatter<df64, 1>(double* y, int p, df64 v, df64, df64) {
  atomicAdd(y + p, to_double(v));
}
// (IQU double-float outputs are weighted in float64 inside k_f3)

template <typename Real>
__device__ __forceinline__ void scatter_mr(typename OutT<Real>::type* y, int p, int q, Real v, Real c, Real s) {
  if constexpr (std::is_same<Real, float>::value) {
    atomicAdd(y + 4LL * p, v);
    atomicAdd(reinterpret_cast<float4*>(y) + q, make_float4(0.0f, v * c, v * s, 0.0f));
  } else {
    atomicAdd(y + 4LL * p, v);
    atomicAdd(y + 4LL * q + 1, v * c);
    atomicAdd(y + 4LL * q + 2, v * s);
  }
}

// A lane seen from one CTA: valid input window positions [in_lo, in_hi),
// kept outputs [out_lo, out_hi), and base pointers already offset by the
// window start so every access is base[n] with a 32-bit window position n.
template <typename Real>
struct LaneView {
  int in_lo, in_hi, out_lo, out_hi;
  const int* pix;
  const float* psi;
  const double2* cs;
  const float4* csd;
  const int2* pw;
  const int* pq;
  const int* pe;
  const int* hb;
  const float* hang;
  const float* htau;
  const void* in;
  const float* in2;  // IN_RESX: d offset by the window start
  void* out;
  int j0;        // on-the-fly pointing: detector sample of window position 0
  float4 dp;     // and the lane's detector offset and orientation
};

template <typename Real, int IN, int OUT>
__device__ __forceinline__ LaneView<Real> lane_view(const OpArgs& a, const Lane& g) {
  LaneView<Real> v;
  const long long ws = g.ws;
  long long lo = g.lo - ws, hi = g.hi - ws;
  lo = lo < 0 ? 0 : (lo > a.M ? a.M : lo);
  hi = hi < lo ? lo : (hi > a.M ? a.M : hi);
  v.in_lo = (int)lo;
  v.in_hi = (int)hi;
  v.out_lo = g.out_lo;
  v.out_hi = g.out_hi;
  v.pix = a.pix + ws;
  v.psi = a.psi + ws;
  v.cs = a.cs64 + ws;
  v.csd = a.csdf + ws;
  v.pw = a.pw + ws;
  v.pq = a.pixq ? a.pixq + ws : nullptr;
  v.pe = a.ext ? a.ext + ws : nullptr;
  v.hb = a.hwp_base ? a.hwp_base + ws : nullptr;
  v.hang = a.hwp_ang ? a.hwp_ang + ws : nullptr;
  v.htau = a.hwp_tau ? a.hwp_tau + ws : nullptr;
  if (a.bore) {
    // windows never leave their interval's detector
    long long dd = a.n_per_det > 0 ? g.lo / a.n_per_det : 0;
    dd = dd < 0 ? 0 : (dd >= a.n_det ? a.n_det - 1 : dd);
    v.j0 = (int)(ws - dd * a.n_per_det);
    v.dp = __ldg(a.det + dd);
  } else {
    v.j0 = 0;
    v.dp = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  v.in2 = IN == IN_RESX ? a.in2 + g.rhs * a.in2_stride + ws : nullptr;
  if (IN == IN_TODF) v.in = static_cast<const float*>(a.in) + g.rhs * a.in_stride + ws;
  else if (IN == IN_TODR) v.in = static_cast<const Real*>(a.in) + g.rhs * a.in_stride + ws;
  else v.in = static_cast<const Real*>(a.in) + g.rhs * a.in_stride;
  typedef typename OutT<Real>::type Out;
  if (OUT == OUT_TOD) v.out = static_cast<Out*>(a.out) + g.rhs * a.out_stride + ws;
  else
    v.out = static_cast<Out*>(a.out) + g.rhs * a.out_stride +
            (a.n_rep > 1 ? (long long)((blockIdx.x + blockIdx.y) % a.n_rep) * a.rep_stride : 0LL);
  return v;
}

__device__ __forceinline__ bool in_range(int n, int lo, int hi) { return (unsigned)(n - lo) < (unsigned)(hi - lo); }

// cos/sin weights of window position n of a lane (psi or cached float64 pair)
template <typename Real>
__device__ __forceinline__ void lane_angle(const LaneView<Real>& L, int n, bool ok, Real& c, Real& s);
template <>
__device__ __forceinline__ void lane_angle<float>(const LaneView<float>& L, int n, bool ok, float& c, float& s) {
  c = ok ? __ldg(L.psi + n) : 0.f;  // the angle; turned into weights after the loads
  s = 0.f;
}
template <>
__device__ __forceinline__ void lane_angle<double>(const LaneView<double>& L, int n, bool ok, double& c, double& s) {
  if (ok) {
    const double2 cs = L.cs[n];
    c = cs.x;
    s = cs.y;
  } else {
    c = s = 0.0;
  }
}
template <>
__device__ __forceinline__ void lane_angle<df64>(const LaneView<df64>& L, int n, bool ok, df64& c, df64& s) {
  if (ok) {
    const float4 cs = L.csd[n];
    c = df64(cs.x, cs.y);
    s = df64(cs.z, cs.w);
  } else {
    c = s = df64();
  }
}
template <typename Real>
__device__ __forceinline__ void finish_angle(Real& c, Real& s) {}

// Pixel and weights' source of window position n of a lane: the float32
// operator reads pixel and angle as one 8-byte pair; the others the pixel and
// their cached cos/sin pairs.
template <typename Real, int NS>
__device__ __forceinline__ void load_pointing(const OpArgs& a, const LaneView<Real>& L, int n, bool ok, int& pp,
                                              Real& c, Real& s) {
  if constexpr (on_the_fly(NS)) {
    float c2 = 0.f, s2 = 0.f;
    int g = -1;
    if (ok)
      g = expand_pointing<std::is_same<Real, float>::value>(a.bore, a.sd, L.j0 + n, L.dp, a.grid_w, a.grid_h,
                                                            polarised(NS), c2, s2);
    pp = g >= 0 ? __ldg(a.g2o + g) : -1;
    c = Real(c2);
    s = Real(s2);
  } else if (polarised(NS) && std::is_same<Real, float>::value) {
    if (ok) {
      const int2 w = __ldg(L.pw + n);
      pp = w.x;
      c = (Real)__int_as_float(w.y);
    } else {
      pp = -1;
      c = Real(0);
    }
    s = Real(0);
  } else {
    pp = ok ? __ldg(L.pix + n) : -1;
    c = s = Real(0);
    if (polarised(NS)) lane_angle<Real>(L, n, ok, c, s);
  }
}
template <>
__device__ __forceinline__ void finish_angle<float>(float& c, float& s) {
  const float psi = c;
  sincos_2psi(psi, s, c);
}

// The memory phases below work in batches: every thread first issues all the
// independent loads of U elements (pointing, then map gathers; or scratch and
// twiddles), and only then consumes them, so each thread keeps U loads in
// flight instead of one.

// Output twiddles exp(-2 pi i m / M) of the four-step transform from two
// small shared tables: lo[b] = w^b for b < L = 2^logL and hi[a] = w^(a L), so
// w^m = hi[m >> logL] * lo[m & (L - 1)] (one complex product, a few ulp).
// Reading them from the M-entry table instead scatters one L2 sector per element.
// The float64 kernels keep reading the M-entry table: on this GPU a float64
// complex product costs more than the scattered load it would replace.
template <typename C>
__device__ __forceinline__ void build_split_twiddles(C* lo, C* hi, const C* twM, int logM, int logL) {
  if constexpr (sizeof(C) == 8) {
    for (int i = threadIdx.x; i < (1 << logL); i += OP_THREADS) lo[i] = twM[i];
    for (int i = threadIdx.x; i < (1 << (logM - logL)); i += OP_THREADS) hi[i] = twM[(long long)i << logL];
  }
}
template <typename C>
__device__ __forceinline__ C split_twiddle(const C* lo, const C* hi, const C* twM, int m, int logL) {
  if constexpr (sizeof(C) != 8) return twM[m];
  else return cmul(hi[m >> logL], lo[m & ((1 << logL) - 1)]);
}
__host__ __device__ inline int split_log(int logM) { return (logM + 1) >> 1; }

// The four-step twiddles of one thread's elements in the column kernels'
// scratch phases.  With 4096 elements per CTA and 256 threads, thread t owns
// elements t + 256 u (u = 0 .. 15): column n1 = n1_0 + (t mod B1) and row
// position p0 + (256 / B1) u, p0 = t / B1, whose bit reversal is
// K0 + brev4(u) (the bits of p0 and of the row step do not overlap).  Its
// twiddles exp(-2 pi i n1 k2 / M) are therefore A B^v, v = brev4(u), with
// A = w^(n1 K0) and B = w^(n1) read once from the split tables: p4[a] = A B^(4a)
// and p1[b] = B^b, so the twiddle of v = 4a + b is p4[a] p1[b] (at most eight
// roundings; float32 only, replacing two scattered table reads per element).
template <typename C>
__device__ __forceinline__ void scratch_twiddles(const C* lo, const C* hi, const C* twM, int n1, int K0, int mask,
                                                 int logL, C (&p4)[4], C (&p1)[4]) {
  const C A = split_twiddle(lo, hi, twM, (n1 * K0) & mask, logL);
  const C B = split_twiddle(lo, hi, twM, n1 & mask, logL);
  const C B2 = cmul(B, B), B4 = cmul(B2, B2), B8 = cmul(B4, B4);
  p1[0].x = 1;
  p1[0].y = 0;
  p1[1] = B;
  p1[2] = B2;
  p1[3] = cmul(B2, B);
  p4[0] = A;
  p4[1] = cmul(A, B4);
  p4[2] = cmul(A, B8);
  p4[3] = cmul(A, cmul(B8, B4));
}
__host__ __device__ constexpr int brev4(int u) {
  return ((u & 1) << 3) | ((u & 2) << 1) | ((u & 4) >> 1) | ((u & 8) >> 3);
}

// Four-step twiddles of one group of the last column pass: positions
// G q + m (G = 2^RL, m < G) of column n1, whose bit reversal over lg bits is
// brev_RL(m) 2^(lg - RL) + brev_(lg-RL)(q); so the twiddle of element m is
// tw[m] = A C^brev_RL(m), A = w^(n1 brev(q)), C = w^(n1 2^(lg - RL)), from two
// split-table reads and products (float32 only).
template <typename C, int RL>
__device__ __forceinline__ void last_group_twiddles(const C* lo, const C* hi, const C* twM, int n1, int q, int lg,
                                                    int mask, int logL, C (&tw)[1 << RL]) {
  const C A = split_twiddle(lo, hi, twM, (n1 * brev_n(q, lg - RL)) & mask, logL);
  const C Cw = split_twiddle(lo, hi, twM, (n1 << (lg - RL)) & mask, logL);
  C p[1 << RL];
  p[0] = A;
  p[1] = cmul(A, Cw);
  if (RL >= 2) {
    const C C2 = cmul(Cw, Cw);
    p[2] = cmul(A, C2);
    p[3] = cmul(p[1], C2);
    if (RL >= 3) {
      const C C4 = cmul(C2, C2);
      p[4] = cmul(A, C4);
      p[5] = cmul(p[1], C4);
      p[6] = cmul(p[2], C4);
      p[7] = cmul(p[3], C4);
    }
  }
#pragma unroll
  for (int m = 0; m < (1 << RL); ++m) tw[m] = p[brev_small<RL>(m)];
}
// Shared entries of the two split tables (none for float64).
__host__ __device__ inline int split_entries(int esz, int logM) {
  return esz == 8 ? (1 << split_log(logM)) + (1 << (logM - split_log(logM))) : 0;
}

// The polarisation weights (cos 2psi, sin 2psi) of each angle exactly as this
// precision's operator kernels form them (a diagnostic of the weights alone).
template <typename Real>
__global__ void k_weights(long long n, const float* __restrict__ psi, Real* c, Real* s) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    Real cc, ss;
    if constexpr (std::is_same<Real, float>::value) {
      sincos_2psi(psi[t], ss, cc);
    } else {
      sincos(2.0 * (double)psi[t], &ss, &cc);
    }
    c[t] = cc;
    s[t] = ss;
  }
}

// ---------------------------------------------------------------- launch shape
// Elements per CTA of the operator kernels (log2; float32 and the float64-size
// types), the column kernels' minimum resident CTAs per SM (float32; float64
// and double-float: three CTAs hold 80 registers a thread, against 96-110 at
// two, and the double-float operator runs 8% faster), and the samples each
// thread keeps in flight in the gather (polarised map input) and the scatter
// (map output) phases.
#ifndef MM_ELOG_F32
#define MM_ELOG_F32 12
#endif
#ifndef MM_MINB_F13
#define MM_MINB_F13 4
#endif
#ifndef MM_MINB_WIDE13
#define MM_MINB_WIDE13 3
#endif
#ifndef MM_U_GATHER
#define MM_U_GATHER 4
#endif
#ifndef MM_U_SCATTER
#define MM_U_SCATTER 4
#endif
// Float32: the outermost radix-8 pass of each transform runs in registers on
// the way into or out of shared memory (1) or inside it like the others (0).
#ifndef MM_REG_PASS
#define MM_REG_PASS 1
#endif
// Float32 column kernels: the last forward (k_f1) and first inverse (k_f3)
// column pass in registers at the scratch write or read (1).
#ifndef MM_REG_LAST
#define MM_REG_LAST 1
#endif
template <typename Real>
__host__ __device__ constexpr int elog() {
  return sizeof(Real) == 4 ? MM_ELOG_F32 : 11;
}

// ---------------------------------------------------------------- runs of one pixel
// In the column kernels' output phases the lanes of each group of B
// consecutive lanes hold B consecutive samples of one window row, and a scan
// that stays in a pixel for several samples gives runs of lanes with the same
// map row.  Each run adds its sum with one atomic from its last lane: a
// segmented inclusive scan over the run (shuffle steps 1, 2, 4, ... < B) instead
// of one atomic per sample.  Every lane of the warp must take part.  (Stopping
// the scan at the warp's longest run measured slower: the straight-line scans
// of a thread's several outputs overlap one another.)
template <int B>
__device__ __forceinline__ void run_geometry(int p, int& start, bool& tail) {
  const int lane = threadIdx.x & 31;
  const int prev = __shfl_up_sync(0xffffffffu, p, 1);
  const bool head = (lane & (B - 1)) == 0 || prev != p;
  const unsigned hm = __ballot_sync(0xffffffffu, head);
  start = 31 - __clz(hm & ((2u << lane) - 1u));
  tail = lane == 31 || ((hm >> (lane + 1)) & 1u);
}
template <int B, typename T>
__device__ __forceinline__ T run_sum(T x, int start) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < B; d <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane - d >= start) x += y;
  }
  return x;
}

// ---------------------------------------------------------------- k_f1
// LG2 > 0 fixes the column length N2 = 2^LG2 at compile time (and with it the
// CTA's column count); LG2 = 0 reads the geometry from the arguments.
template <typename Real, int NS, int IN, int LG2>
__global__ void __launch_bounds__(256, sizeof(Real) == 4 ? MM_MINB_F13 : MM_MINB_WIDE13) k_f1(OpArgs a) {
  typedef typename CxT<Real>::type C;
  constexpr int ELOG = elog<Real>();
  const int logN2 = LG2 ? LG2 : a.logN2;
  const int logB1 = LG2 ? ELOG - LG2 : a.logB1;
  const int N2 = 1 << logN2, B1 = 1 << logB1;
  const int tl = blockIdx.y;
  const Tile* T = a.tiles + a.tile0 + tl;
  if (skip_tile(a, T)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int SW = LG2 ? lay_sw(sizeof(C), LG2, true) : (sizeof(C) == 16 ? 0 : 1);
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int rs = lay_rs(sizeof(C), logN2, true);
  C* tw = buf + B1 * rs;
  const int logM = a.logN1 + logN2, logL = split_log(logM);
  C* tlo = tw + N2;
  C* thi = tlo + (1 << logL);
  const C* twM = static_cast<const C*>(a.tw);
  build_pass_twiddles(tw, logN2, twM, a.N1);
  build_split_twiddles(tlo, thi, twM, logM, logL);
  LaneView<Real> L[2];
  L[0] = lane_view<Real, IN, OUT_MAP>(a, T->l[0]);
  L[1] = lane_view<Real, IN, OUT_MAP>(a, T->l[1]);
  const int n1_0 = blockIdx.x * B1;
  const int total = B1 << logN2;
  constexpr int bd = OP_THREADS;
  constexpr int U = (gathers(IN) && polarised(NS)) ? MM_U_GATHER : 8;
  // the input values of elements ee[0 .. U-1] (lane 0, lane 1), all loads of
  // the batch issued before any is consumed
  auto gather_batch = [&](const int (&ee)[U], Real (&v)[2][U]) {
    int nn[U];
    bool ok[2][U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = ee[u];
      nn[u] = n1_0 + (e & (B1 - 1)) + ((e >> logB1) << a.logN1);
#pragma unroll
      for (int l = 0; l < 2; ++l) ok[l][u] = e < total && in_range(nn[u], L[l].in_lo, L[l].in_hi);
    }
    if (!gathers(IN)) {
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          if (IN == IN_TODF)
            v[l][u] = ok[l][u] ? (Real)__ldg(static_cast<const float*>(L[l].in) + nn[u]) : Real(0);
          else
            v[l][u] = ok[l][u] ? static_cast<const Real*>(L[l].in)[nn[u]] : Real(0);
        }
    } else {
      int pp[2][U], qq[2][U];
      Real cc[2][U], ss[2][U];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          load_pointing<Real, NS>(a, L[l], nn[u], ok[l][u], pp[l][u], cc[l][u], ss[l][u]);
          if constexpr (NS == NS_MR || extended(NS)) {
            const int* qp = NS == NS_MR ? L[l].pq : L[l].pe;
            qq[l][u] = (ok[l][u] && qp) ? __ldg(qp + nn[u]) : -1;
          }
        }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          Real c = cc[l][u], sn = ss[l][u];
          if (polarised(NS) && !on_the_fly(NS)) finish_angle<Real>(c, sn);
          const Real* x = static_cast<const Real*>(L[l].in);
          if constexpr (NS == NS_MR) {
            v[l][u] = pp[l][u] >= 0 ? gather_mr<Real>(x, pp[l][u], qq[l][u], c, sn) : Real(0);
          } else {
            v[l][u] = pp[l][u] >= 0 ? gather<Real, map_ns(NS)>(x, pp[l][u], c, sn) : Real(0);
            if constexpr (extended(NS)) {   // + the extra column's amplitude (slot 0 of its row)
              if (pp[l][u] >= 0 && qq[l][u] >= 0) v[l][u] += x[(long long)qq[l][u] * (map_ns(NS) == 3 ? 4 : 1)];
              if (pp[l][u] >= 0 && L[l].hb) {   // + the half-wave-plate term
                const int hb = __ldg(L[l].hb + nn[u]);
                if (hb >= 0)
                  v[l][u] += hwp_gather<Real>(x, hb, map_ns(NS) == 3 ? 4 : 1, __ldg(L[l].hang + nn[u]),
                                              __ldg(L[l].htau + nn[u]));
              }
            }
          }
        }
    }
    if constexpr (IN == IN_RESX) {   // d - A x (flagged samples: rows of A are zero)
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int l = 0; l < 2; ++l)
          if (ok[l][u]) v[l][u] = Real(__ldg(L[l].in2 + nn[u])) - v[l][u];
    }
  };
  // float32 with compile-time geometry: thread t's 16 elements t + 256 u are
  // the two radix-8 groups (bases p0 and p0 + N2/16, stride N2/8) of the first
  // column pass, which therefore runs in registers before the first store
  constexpr bool REG1 = sizeof(C) == 8 && LG2 >= 4 && MM_REG_PASS && ELOG == 12 && OP_THREADS == 256 &&
                        (U == 4 || U == 8);
  if constexpr (REG1) {
    constexpr int lgh = LG2 - 3;
    const int jc = threadIdx.x & (B1 - 1), p0 = threadIdx.x >> logB1;
    __syncthreads();  // the pass twiddle tables
#pragma unroll 1
    for (int G = 0; G < 2; ++G) {
      C gv[8];
#pragma unroll
      for (int b = 0; b < 8 / U; ++b) {
        int ee[U];
        Real v[2][U];
#pragma unroll
        for (int k = 0; k < U; ++k) ee[k] = threadIdx.x + (2 * (U * b + k) + G) * bd;
        gather_batch(ee, v);
#pragma unroll
        for (int k = 0; k < U; ++k) {
          gv[U * b + k].x = v[0][k];
          gv[U * b + k].y = v[1][k];
        }
      }
      const int base = p0 + (G << (lgh - 1));
      reg_pass8<C, false>(gv, tw, LG2, base);
#pragma unroll
      for (int m = 0; m < 8; ++m) buf[jc * rs + swz<SW>(base + (m << lgh))] = gv[m];
    }
  } else {
    for (int e0 = threadIdx.x; e0 < total; e0 += bd * U) {
      int ee[U];
      Real v[2][U];
#pragma unroll
      for (int u = 0; u < U; ++u) ee[u] = e0 + u * bd;
      gather_batch(ee, v);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = ee[u];
        if (e < total) {
          C z;
          z.x = v[0][u];
          z.y = v[1][u];
          buf[(e & (B1 - 1)) * rs + swz<SW>(e >> logB1)] = z;
        }
      }
    }
  }
  __syncthreads();
  // float32 with compile-time geometry: the last column pass (radix 4 or 8 on
  // consecutive elements, no twiddles) runs in registers and feeds the
  // scratch write directly
  constexpr int RL = LG2 > 0 ? LG2 - last_pass_start(LG2) : 0;
  constexpr bool REGL = REG1 && MM_REG_LAST && (RL == 2 || RL == 3) && last_pass_start(LG2) >= 6;
  fft_rows<C, false, SW>(buf, B1, rs, logN2, tw, REG1 ? 3 : 0, REGL ? last_pass_start(LG2) : -1);
  C* sc = static_cast<C*>(a.scratch) + (long long)tl * a.M;
  const int mask = a.M - 1;
  if constexpr (REGL) {
    constexpr int G = 1 << RL;
    const int j = threadIdx.x & (B1 - 1);
#pragma unroll 1
    for (int q = threadIdx.x >> logB1; q < (N2 >> RL); q += bd >> logB1) {
      C v[G], w[G];
#pragma unroll
      for (int m = 0; m < G; ++m) v[m] = buf[j * rs + swz<SW>(G * q + m)];
      reg_pass_last<C, RL, false>(v);
      last_group_twiddles<C, RL>(tlo, thi, twM, n1_0 + j, q, LG2, mask, logL, w);
#pragma unroll
      for (int m = 0; m < G; ++m) sc[(long long)(G * q + m) * a.N1 + n1_0 + j] = cmul(v[m], w[m]);
    }
  } else if constexpr (sizeof(C) == 8 && LG2 > 0 && MM_TW_POWERS && ELOG == 12 && OP_THREADS == 256) {
    const int j = threadIdx.x & (B1 - 1), p0 = threadIdx.x >> logB1;
    C p4[4], p1[4];
    scratch_twiddles(tlo, thi, twM, n1_0 + j, brev_n(p0, logN2), mask, logL, p4, p1);
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int v = brev4(u), pos = p0 + (u << (8 - logB1));
      sc[(long long)pos * a.N1 + n1_0 + j] = cmul(buf[j * rs + swz<SW>(pos)], cmul(p4[v >> 2], p1[v & 3]));
    }
  } else {
#pragma unroll 4
    for (int e = threadIdx.x; e < total; e += bd) {
      const int j = e & (B1 - 1), pos = e >> logB1;
      const C w = split_twiddle(tlo, thi, twM, ((n1_0 + j) * brev_n(pos, logN2)) & mask, logL);
      sc[(long long)pos * a.N1 + n1_0 + j] = cmul(buf[j * rs + swz<SW>(pos)], w);
    }
  }
}

// ---------------------------------------------------------------- k_f2
// LG1 > 0 fixes the row length N1 = 2^LG1 at compile time.
template <typename Real, int LG1>
__global__ void __launch_bounds__(256, sizeof(Real) == 4 ? 4 : 2) k_f2(OpArgs a) {
  typedef typename CxT<Real>::type C;
  constexpr int ELOG = elog<Real>();
  const int logN1 = LG1 ? LG1 : a.logN1;
  const int N1 = 1 << logN1;
  const int B2 = LG1 ? (1 << (ELOG - LG1)) : a.B2;
  const int tl = blockIdx.y;
  const Tile* T = a.tiles + a.tile0 + tl;
  if (skip_tile(a, T)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int SW = LG1 ? lay_sw(sizeof(C), LG1, false) : 1;
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int rs = lay_rs(sizeof(C), logN1, false);
  C* tw = buf + B2 * rs;
  const C* twM = static_cast<const C*>(a.tw);
  build_pass_twiddles(tw, logN1, twM, a.N2);
  const int filt = T->filter;
  const int pos0 = blockIdx.x * B2;
  C* sc = static_cast<C*>(a.scratch) + (long long)tl * a.M + (long long)pos0 * N1;
  const int total = B2 << logN1;
  constexpr int bd = OP_THREADS;
  const Real* H = static_cast<const Real*>(a.H) + (long long)filt * a.M + (long long)pos0 * N1;
  auto Hrow = [H, N1](int row) { return H + (long long)row * N1; };
  if constexpr (sizeof(C) == 8 && LG1 >= 4 && MM_REG_PASS && ELOG == 12 && OP_THREADS == 256) {
    // float32: the first forward and the last inverse pass in registers,
    // straight from and to the scratch.  Thread t owns the groups g = t and
    // t + 256 (row g / (N1/8), elements j + m N1/8, j = g mod N1/8); a warp's
    // loads and stores of one m cover 32 consecutive elements of one row.
    constexpr int lgh = LG1 - 3;
    __syncthreads();  // the pass twiddle tables
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int g = threadIdx.x + h * bd, row = g >> lgh, j = g & ((1 << lgh) - 1);
      C v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = sc[(row << LG1) + j + (m << lgh)];
      reg_pass8<C, false>(v, tw, LG1, j);
#pragma unroll
      for (int m = 0; m < 8; ++m) buf[row * rs + swz<SW>(j + (m << lgh))] = v[m];
    }
    __syncthreads();
    fft_rows_filter<C, SW>(buf, B2, rs, logN1, tw, Hrow, 3);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int g = threadIdx.x + h * bd, row = g >> lgh, j = g & ((1 << lgh) - 1);
      C v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = buf[row * rs + swz<SW>(j + (m << lgh))];
      reg_pass8<C, true>(v, tw, LG1, j);
#pragma unroll
      for (int m = 0; m < 8; ++m) sc[(row << LG1) + j + (m << lgh)] = v[m];
    }
  } else {
    for (int e0 = threadIdx.x; e0 < total; e0 += bd * 8) {
      C v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (e0 + u * bd < total) v[u] = sc[e0 + u * bd];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * bd;
        if (e < total) buf[(e >> logN1) * rs + swz<SW>(e & (N1 - 1))] = v[u];
      }
    }
    __syncthreads();
    fft_rows_filter<C, SW>(buf, B2, rs, logN1, tw, Hrow);
    for (int e = threadIdx.x; e < total; e += bd) sc[e] = buf[(e >> logN1) * rs + swz<SW>(e & (N1 - 1))];
  }
}

// ---------------------------------------------------------------- k_f3
template <typename Real, int NS, int OUT, int LG2>
__global__ void __launch_bounds__(256, sizeof(Real) == 4 ? MM_MINB_F13 : MM_MINB_WIDE13) k_f3(OpArgs a) {
  typedef typename CxT<Real>::type C;
  constexpr int ELOG = elog<Real>();
  const int logN2 = LG2 ? LG2 : a.logN2;
  const int logB1 = LG2 ? ELOG - LG2 : a.logB1;
  const int N2 = 1 << logN2, B1 = 1 << logB1;
  const int tl = blockIdx.y;
  const Tile* T = a.tiles + a.tile0 + tl;
  if (skip_tile(a, T)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int SW = LG2 ? lay_sw(sizeof(C), LG2, true) : (sizeof(C) == 16 ? 0 : 1);
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int rs = lay_rs(sizeof(C), logN2, true);
  C* tw = buf + B1 * rs;
  const int logM = a.logN1 + logN2, logL = split_log(logM);
  C* tlo = tw + N2;
  C* thi = tlo + (1 << logL);
  const C* twM = static_cast<const C*>(a.tw);
  build_pass_twiddles(tw, logN2, twM, a.N1);
  build_split_twiddles(tlo, thi, twM, logM, logL);
  // half-wave-plate sums of the CTA, per tile lane (extended pointing only)
  constexpr bool HWP = extended(NS) && OUT == OUT_MAP;
  __shared__ typename OutT<Real>::type hacc[HWP ? 64 : 1];
  __shared__ int hgrp[2];
  if (HWP) {
    for (int i = threadIdx.x; i < 64; i += OP_THREADS) hacc[i] = 0;
    if (threadIdx.x < 2) hgrp[threadIdx.x] = -1;
  }
  __syncthreads();
  LaneView<Real> L[2];
  L[0] = lane_view<Real, IN_MAPX, OUT>(a, T->l[0]);
  L[1] = lane_view<Real, IN_MAPX, OUT>(a, T->l[1]);
  const int n1_0 = blockIdx.x * B1;
  const int total = B1 << logN2;
  constexpr int bd = OP_THREADS;
  const C* sc = static_cast<const C*>(a.scratch) + (long long)tl * a.M;
  const int mask = a.M - 1;
  // float32 with compile-time geometry: the first inverse column pass (radix
  // 4 or 8 on consecutive elements, no twiddles) runs in registers on the
  // groups read straight from the scratch (see k_f1)
  constexpr int RL = LG2 > 0 ? LG2 - last_pass_start(LG2) : 0;
  constexpr bool REGH = sizeof(C) == 8 && LG2 >= 4 && MM_REG_PASS && MM_REG_LAST && ELOG == 12 &&
                        OP_THREADS == 256 && (RL == 2 || RL == 3) && last_pass_start(LG2) >= 6;
  if constexpr (REGH) {
    constexpr int G = 1 << RL;
    const int j = threadIdx.x & (B1 - 1);
#pragma unroll 2
    for (int q = threadIdx.x >> logB1; q < (N2 >> RL); q += bd >> logB1) {
      C v[G], w[G];
#pragma unroll
      for (int m = 0; m < G; ++m) v[m] = sc[(long long)(G * q + m) * a.N1 + n1_0 + j];
      last_group_twiddles<C, RL>(tlo, thi, twM, n1_0 + j, q, LG2, mask, logL, w);
#pragma unroll
      for (int m = 0; m < G; ++m) v[m] = cmulc(v[m], w[m]);
      reg_pass_last<C, RL, true>(v);
#pragma unroll
      for (int m = 0; m < G; ++m) buf[j * rs + swz<SW>(G * q + m)] = v[m];
    }
  } else if constexpr (sizeof(C) == 8 && LG2 > 0 && MM_TW_POWERS && ELOG == 12 && OP_THREADS == 256) {
    const int j = threadIdx.x & (B1 - 1), p0 = threadIdx.x >> logB1;
    C p4[4], p1[4];
    scratch_twiddles(tlo, thi, twM, n1_0 + j, brev_n(p0, logN2), mask, logL, p4, p1);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      C v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = sc[(long long)(p0 + ((8 * h + k) << (8 - logB1))) * a.N1 + n1_0 + j];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int u = 8 * h + k, w = brev4(u), pos = p0 + (u << (8 - logB1));
        buf[j * rs + swz<SW>(pos)] = cmulc(v[k], cmul(p4[w >> 2], p1[w & 3]));
      }
    }
  } else {
    for (int e0 = threadIdx.x; e0 < total; e0 += bd * 8) {
      C v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * bd;
        if (e < total) v[u] = sc[(long long)(e >> logB1) * a.N1 + n1_0 + (e & (B1 - 1))];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * bd;
        if (e < total) {
          const int n1 = n1_0 + (e & (B1 - 1)), pos = e >> logB1;
          const C w = split_twiddle(tlo, thi, twM, (n1 * brev_n(pos, logN2)) & mask, logL);
          buf[(e & (B1 - 1)) * rs + swz<SW>(pos)] = cmulc(v[u], w);
        }
      }
    }
  }
  __syncthreads();
  constexpr int U = OUT == OUT_MAP ? MM_U_SCATTER : 8;
  // lanes per group of consecutive samples (compile-time geometry only)
  constexpr int RUNB = LG2 > 0 ? ((1 << (ELOG - LG2)) < 32 ? (1 << (ELOG - LG2)) : 32) : 0;
  // the outputs of elements ee[0 .. U-1] with values val (lane 0, lane 1)
  auto scatter_batch = [&](const int (&eidx)[U], const Real (&val)[2][U]) {
    int nn[U];
    bool ok[2][U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = eidx[u];
      nn[u] = n1_0 + (e & (B1 - 1)) + ((e >> logB1) << a.logN1);
#pragma unroll
      for (int l = 0; l < 2; ++l) ok[l][u] = e < total && in_range(nn[u], L[l].out_lo, L[l].out_hi);
    }
    if (OUT == OUT_TOD) {
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int l = 0; l < 2; ++l)
          if (ok[l][u]) static_cast<typename OutT<Real>::type*>(L[l].out)[nn[u]] = to_out(val[l][u]);
    } else if constexpr (std::is_same<Real, df64>::value && polarised(NS)) {
      // double-float: round the value to float64 once and weight it with the
      // float64 (cos, sin) pair (5 float64 operations per sample, not 9)
      int pp[2][U], qq[2][U], ee[2][U];
      double2 cs[2][U];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          if constexpr (on_the_fly(NS)) {
            df64 c, sn;
            load_pointing<Real, NS>(a, L[l], nn[u], ok[l][u], pp[l][u], c, sn);
            cs[l][u] = make_double2(to_double(c), to_double(sn));
          } else {
            pp[l][u] = ok[l][u] ? __ldg(L[l].pix + nn[u]) : -1;
            cs[l][u] = ok[l][u] ? L[l].cs[nn[u]] : make_double2(0.0, 0.0);
          }
          if constexpr (NS == NS_MR) qq[l][u] = ok[l][u] ? __ldg(L[l].pq + nn[u]) : -1;
          else qq[l][u] = pp[l][u];
          if constexpr (extended(NS)) ee[l][u] = (ok[l][u] && L[l].pe) ? __ldg(L[l].pe + nn[u]) : -1;
        }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          if (pp[l][u] < 0) continue;
          double* y = static_cast<double*>(L[l].out);
          const double v = to_double(val[l][u]);
          atomicAdd(y + 4LL * pp[l][u], v);
          atomicAdd(y + 4LL * qq[l][u] + 1, v * cs[l][u].x);
          atomicAdd(y + 4LL * qq[l][u] + 2, v * cs[l][u].y);
          if constexpr (extended(NS)) {
            if (ee[l][u] >= 0) atomic_add_warp(y, 4LL * ee[l][u], v);
          }
        }
    } else {
      int pp[2][U], qq[2][U];
      Real cc[2][U], ss[2][U];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          load_pointing<Real, NS>(a, L[l], nn[u], ok[l][u], pp[l][u], cc[l][u], ss[l][u]);
          if constexpr (NS == NS_MR || extended(NS)) {
            const int* qp = NS == NS_MR ? L[l].pq : L[l].pe;
            qq[l][u] = (ok[l][u] && qp) ? __ldg(qp + nn[u]) : -1;
          }
        }
      // float32: one atomic per run of samples in one pixel (in float64 and
      // double-float the shuffles of the partial sums cost more than the
      // atomics they save)
      if constexpr (RUNB > 0 && (NS == 1 || NS == 3) && std::is_same<Real, float>::value) {
        if (a.runs) {
#pragma unroll
          for (int u = 0; u < U; ++u)
#pragma unroll
            for (int l = 0; l < 2; ++l) {
              int start;
              bool tail;
              run_geometry<RUNB>(pp[l][u], start, tail);
              const float v = pp[l][u] >= 0 ? val[l][u] : 0.0f;
              const float s0 = run_sum<RUNB>(v, start);
              if constexpr (NS == 1) {
                if (tail && pp[l][u] >= 0) atomicAdd(static_cast<float*>(L[l].out) + pp[l][u], s0);
              } else {
                float c = cc[l][u], sn = ss[l][u];
                finish_angle<float>(c, sn);
                const float s1 = run_sum<RUNB>(v * c, start), s2 = run_sum<RUNB>(v * sn, start);
                if (tail && pp[l][u] >= 0)
                  atomicAdd(reinterpret_cast<float4*>(L[l].out) + pp[l][u], make_float4(s0, s1, s2, 0.0f));
              }
            }
          return;
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          if (pp[l][u] < 0) continue;
          if constexpr (extended(NS)) {   // the extra column's share (slot 0 of its row)
            typedef typename OutT<Real>::type Out;
            if (qq[l][u] >= 0)
              atomic_add_warp(static_cast<Out*>(L[l].out), (long long)qq[l][u] * (map_ns(NS) == 3 ? 4 : 1),
                              (Out)to_out(val[l][u]));
          }
          Real c = cc[l][u], sn = ss[l][u];
          if (polarised(NS) && !on_the_fly(NS)) finish_angle<Real>(c, sn);
          if constexpr (NS == NS_MR)
            scatter_mr<Real>(static_cast<typename OutT<Real>::type*>(L[l].out), pp[l][u], qq[l][u], val[l][u], c, sn);
          else
            scatter<Real, map_ns(NS)>(static_cast<typename OutT<Real>::type*>(L[l].out), pp[l][u], val[l][u], c, sn);
        }
    }
    if constexpr (extended(NS) && OUT == OUT_MAP) {
      if (a.hwp_base) {   // half-wave-plate parameters, one converged warp at a time
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int l = 0; l < 2; ++l)
            hwp_scatter_warp<Real>(hacc + 32 * l, hgrp + l, L[l].pix, L[l].hb, L[l].hang, L[l].htau, nn[u],
                                   ok[l][u], val[l][u]);
      }
    }
  };
  // float32 with compile-time geometry: the last inverse column pass runs in
  // registers on each thread's two radix-8 groups (see k_f1) before their outputs
  constexpr bool REG3 = sizeof(C) == 8 && LG2 >= 4 && MM_REG_PASS && ELOG == 12 && OP_THREADS == 256 &&
                        (U == 4 || U == 8);
  fft_rows<C, true, SW>(buf, B1, rs, logN2, tw, REG3 ? 3 : 0, REGH ? last_pass_start(LG2) : -1);
  if constexpr (REG3) {
    constexpr int lgh = LG2 - 3;
    const int jc = threadIdx.x & (B1 - 1), p0 = threadIdx.x >> logB1;
#pragma unroll 1
    for (int G = 0; G < 2; ++G) {
      const int base = p0 + (G << (lgh - 1));
      C gv[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) gv[m] = buf[jc * rs + swz<SW>(base + (m << lgh))];
      reg_pass8<C, true>(gv, tw, LG2, base);
#pragma unroll
      for (int b = 0; b < 8 / U; ++b) {
        int ee[U];
        Real val[2][U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
          ee[k] = threadIdx.x + (2 * (U * b + k) + G) * bd;
          val[0][k] = gv[U * b + k].x;
          val[1][k] = gv[U * b + k].y;
        }
        scatter_batch(ee, val);
      }
    }
  } else {
    for (int e0 = threadIdx.x; e0 < total; e0 += bd * U) {
      int ee[U];
      Real val[2][U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * bd;
        ee[u] = e;
        C z;
        z.x = z.y = 0;
        if (e < total) z = buf[(e & (B1 - 1)) * rs + swz<SW>(e >> logB1)];
        val[0][u] = z.x;
        val[1][u] = z.y;
      }
      scatter_batch(ee, val);
    }
  }
  if constexpr (HWP) {
    if (a.hwp_base) {
      __syncthreads();
      for (int l = 0; l < 2; ++l)
        hwp_flush(static_cast<typename OutT<Real>::type*>(L[l].out), map_ns(NS) == 3 ? 4 : 1, hacc + 32 * l,
                  hgrp + l, 1);
    }
  }
}


// ---------------------------------------------------------------- k_diag
// White noise (one filter lag, e.g. destriping runs, Section 6 item 3): N^-1
// is f(0) of the interval's filter times the identity, so the operator is a
// single pass, gather -> weight -> scatter, with no windows and no FFT.  One
// CTA per run of samples of one interval.
template <typename Real, int NS>
__device__ __forceinline__ Real sample_gather(const OpArgs& a, const LaneView<Real>& L, int n) {
  int pp;
  Real c, sn;
  load_pointing<Real, NS>(a, L, n, true, pp, c, sn);
  if (pp < 0) return Real(0);
  if (polarised(NS) && !on_the_fly(NS)) finish_angle<Real>(c, sn);
  const Real* x = static_cast<const Real*>(L.in);
  if constexpr (NS == NS_MR) {
    return gather_mr<Real>(x, pp, __ldg(L.pq + n), c, sn);
  } else {
    Real v = gather<Real, map_ns(NS)>(x, pp, c, sn);
    if constexpr (extended(NS)) {
      const int e = L.pe ? __ldg(L.pe + n) : -1;
      if (e >= 0) v += x[(long long)e * (map_ns(NS) == 3 ? 4 : 1)];
      const int hb = L.hb ? __ldg(L.hb + n) : -1;
      if (hb >= 0) v += hwp_gather<Real>(x, hb, map_ns(NS) == 3 ? 4 : 1, __ldg(L.hang + n), __ldg(L.htau + n));
    }
    return v;
  }
}

template <typename Real, int NS>
__device__ __forceinline__ void sample_scatter(const OpArgs& a, const LaneView<Real>& L, int n, Real val) {
  typedef typename OutT<Real>::type Out;
  int pp;
  Real c, sn;
  load_pointing<Real, NS>(a, L, n, true, pp, c, sn);
  if (pp < 0) return;
  Out* y = static_cast<Out*>(L.out);
  if constexpr (extended(NS)) {
    const int e = L.pe ? __ldg(L.pe + n) : -1;
    if (e >= 0) atomic_add_warp(y, (long long)e * (map_ns(NS) == 3 ? 4 : 1), (Out)to_out(val));
  }
  if constexpr (std::is_same<Real, df64>::value && polarised(NS)) {
    // as k_f3: the value rounded to float64 once, weighted by the float64 pair
    double2 cs;
    if constexpr (on_the_fly(NS)) cs = make_double2(to_double(c), to_double(sn));
    else cs = L.cs[n];
    const int q = NS == NS_MR ? __ldg(L.pq + n) : pp;
    const double v = to_double(val);
    atomicAdd(y + 4LL * pp, v);
    atomicAdd(y + 4LL * q + 1, v * cs.x);
    atomicAdd(y + 4LL * q + 2, v * cs.y);
  } else {
    if (polarised(NS) && !on_the_fly(NS)) finish_angle<Real>(c, sn);
    if constexpr (NS == NS_MR) scatter_mr<Real>(y, pp, __ldg(L.pq + n), val, c, sn);
    else scatter<Real, map_ns(NS)>(y, pp, val, c, sn);
  }
}

// HWP: the instance for plans with half-wave-plate parameters (extended
// pointing); the others keep the plain loop.
template <typename Real, int NS, int IN, int OUT, bool HWP>
__global__ void __launch_bounds__(256) k_diag(OpArgs a, const DiagItem* __restrict__ items, const double* f0) {
  if (a.skip && *a.skip) return;
  const DiagItem it = items[blockIdx.x];
  Lane g;
  g.ws = it.lo;
  g.lo = it.lo;
  g.hi = it.hi;
  g.out_lo = 0;
  g.out_hi = (int)(it.hi - it.lo);
  g.rhs = 0;
  const LaneView<Real> L = lane_view<Real, IN, OUT>(a, g);
  const Real w0 = Real(f0[it.filter]);
  const int len = (int)(it.hi - it.lo);
  if constexpr (!HWP) {
    for (int n = threadIdx.x; n < len; n += blockDim.x) {
      Real v;
      if (IN == IN_MAPX) v = sample_gather<Real, NS>(a, L, n);
      else if (IN == IN_RESX) v = Real(__ldg(L.in2 + n)) - sample_gather<Real, NS>(a, L, n);
      else if (IN == IN_TODF) v = (Real)__ldg(static_cast<const float*>(L.in) + n);
      else v = static_cast<const Real*>(L.in)[n];
      v = v * w0;
      if (OUT == OUT_TOD) static_cast<typename OutT<Real>::type*>(L.out)[n] = to_out(v);
      else sample_scatter<Real, NS>(a, L, n, v);
    }
  } else {
    __shared__ typename OutT<Real>::type hacc[32];
    __shared__ int hgrp[1];
    if (threadIdx.x < 32) hacc[threadIdx.x] = 0;
    if (threadIdx.x == 0) hgrp[0] = -1;
    __syncthreads();
    // whole-block rounds, so every warp stays converged for the half-wave-plate scatter
    for (int n0 = 0; n0 < len; n0 += blockDim.x) {
      const int n = n0 + threadIdx.x;
      const bool in = n < len;
      Real v = Real(0);
      if (in) {
        if (IN == IN_MAPX) v = sample_gather<Real, NS>(a, L, n);
        else if (IN == IN_RESX) v = Real(__ldg(L.in2 + n)) - sample_gather<Real, NS>(a, L, n);
        else if (IN == IN_TODF) v = (Real)__ldg(static_cast<const float*>(L.in) + n);
        else v = static_cast<const Real*>(L.in)[n];
        v = v * w0;
        sample_scatter<Real, NS>(a, L, n, v);
      }
      hwp_scatter_warp<Real>(hacc, hgrp, L.pix, L.hb, L.hang, L.htau, n, in, v);
    }
    __syncthreads();
    hwp_flush(static_cast<typename OutT<Real>::type*>(L.out), map_ns(NS) == 3 ? 4 : 1, hacc, hgrp, 1);
  }
}

// out += the sum of the map replicas, which are left zero for the next application
template <typename Out>
__global__ void k_rep_reduce(Out* rep, int n_rep, long long stride, Out* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    Out acc = Out(0);
    for (int k = 0; k < n_rep; ++k) {
      acc += rep[k * stride + i];
      rep[k * stride + i] = Out(0);
    }
    out[i] += acc;
  }
}

template <typename Real>
inline int elems_per_cta() {
  return 1 << elog<Real>();
}

template <typename Real>
void geometry(const Plan* p, int& B1, int& B2) {
  const int E = elems_per_cta<Real>();
  B1 = E / p->N2;
  if (B1 < 1) B1 = 1;
  if (B1 > p->N1) B1 = p->N1;
  B2 = E / p->N1;
  if (B2 < 1) B2 = 1;
  if (B2 > p->N2) B2 = p->N2;
}

template <typename Real>
size_t smem_f13(const Plan* p) {
  int B1, B2;
  geometry<Real>(p, B1, B2);
  typedef typename CxT<Real>::type C;
  return (size_t)(B1 * lay_rs(sizeof(C), p->logN2, true) + p->N2 + split_entries(sizeof(C), p->logN1 + p->logN2)) *
         sizeof(C);
}
template <typename Real>
size_t smem_f2(const Plan* p) {
  int B1, B2;
  geometry<Real>(p, B1, B2);
  return (size_t)(B2 * lay_rs(sizeof(typename CxT<Real>::type), p->logN1, false) + p->N1) *
         sizeof(typename CxT<Real>::type);
}

typedef void (*OpKernel)(OpArgs);

// Raise a kernel's dynamic shared-memory limit when a plan needs more than it
// was last given (once per kernel instance and size; host-side bookkeeping).
cudaError_t set_smem(OpKernel kernel, size_t bytes) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, size_t>> done;
  std::lock_guard<std::mutex> lk(mu);
  for (auto& d : done)
    if (d.first == (const void*)kernel) {
      if (d.second >= bytes) return cudaSuccess;
      d.second = bytes;
      return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    }
  done.push_back({(const void*)kernel, bytes});
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// The three operator kernels for a plan: instances with compile-time FFT
// geometry for the common sizes, the generic instances otherwise.
struct OpKernels {
  OpKernel f1, f2, f3;
};

template <typename Real, int NS, int IN, int OUT>
OpKernels pick_kernels(const Plan* p) {
  OpKernels k;
  // the T on-the-fly and extended-pointing modes keep only the generic column
  // kernels (fewer instances to compile)
  constexpr bool generic_only = NS == NS_OTF_T || extended(NS);
  if constexpr (generic_only) {
    k.f1 = k_f1<Real, NS, IN, 0>;
    k.f3 = k_f3<Real, NS, OUT, 0>;
  } else {
    switch (p->logN2) {
      case 7: k.f1 = k_f1<Real, NS, IN, 7>; k.f3 = k_f3<Real, NS, OUT, 7>; break;
      case 8: k.f1 = k_f1<Real, NS, IN, 8>; k.f3 = k_f3<Real, NS, OUT, 8>; break;
      case 9: k.f1 = k_f1<Real, NS, IN, 9>; k.f3 = k_f3<Real, NS, OUT, 9>; break;
      case 10: k.f1 = k_f1<Real, NS, IN, 10>; k.f3 = k_f3<Real, NS, OUT, 10>; break;
      default: k.f1 = k_f1<Real, NS, IN, 0>; k.f3 = k_f3<Real, NS, OUT, 0>; break;
    }
  }
  switch (p->logN1) {
    case 6: k.f2 = k_f2<Real, 6>; break;
    case 7: k.f2 = k_f2<Real, 7>; break;
    case 8: k.f2 = k_f2<Real, 8>; break;
    case 9: k.f2 = k_f2<Real, 9>; break;
    case 10: k.f2 = k_f2<Real, 10>; break;
    default: k.f2 = k_f2<Real, 0>; break;
  }
  return k;
}

// ---------------------------------------------------------------- ordered sums (deterministic plans)
// A^T w summed row by row in a fixed order: one warp per observed row walks
// the row's samples in ascending order (lane k takes samples k, k + 32, ...,
// then a fixed butterfly adds the lanes), so every application gives the same
// bits.  w: the weighted timestream N^-1 A x of each right-hand side
// (blockIdx.y), w_stride apart; the row's sums are added into out.  The
// weights are formed as the atomic scatter forms them: float32 from psi by
// sincos_2psi, float64 and double-float from the float64 pair cs64.
template <typename Real, int NS>
__global__ void __launch_bounds__(256) k_segsum(const typename OutT<Real>::type* __restrict__ w, long long w_stride,
                                                const int* __restrict__ ptr, const int* __restrict__ idx, int n_obs,
                                                const float* __restrict__ psi, const double2* __restrict__ cs64,
                                                typename OutT<Real>::type* out, long long out_stride, const int* skip,
                                                int skip_stride) {
  typedef typename OutT<Real>::type Out;
  const int r = blockIdx.y;
  if (skip && (skip_stride == 0 ? *skip != 0 : skip[r * skip_stride] != 0)) return;
  w += r * w_stride;
  out += r * out_stride;
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n_obs; p += nw) {
    const int b = ptr[p], e = ptr[p + 1];
    Out a0 = Out(0), a1 = Out(0), a2 = Out(0);
    for (int k = b + lane; k < e; k += 32) {
      const int t = __ldg(idx + k);
      const Out v = w[t];
      if constexpr (NS == 1) {
        a0 += v;
      } else {
        Out c, sn;
        if constexpr (std::is_same<Real, float>::value) {
          sincos_2psi(__ldg(psi + t), sn, c);
        } else {
          const double2 cs = cs64[t];
          c = cs.x;
          sn = cs.y;
        }
        a0 += v;
        a1 += v * c;
        a2 += v * sn;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      if (NS == 3) {
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
      }
    }
    if (lane == 0) {
      if (NS == 1) {
        out[p] += a0;
      } else {
        Out* q = out + 4LL * p;
        q[0] += a0;
        q[1] += a1;
        q[2] += a2;
      }
    }
  }
}

template <typename Real, int NS, int IN, int OUT>
madmap_status launch_all(Plan* p, const void* in, void* out, long long in_stride, long long out_stride,
                         int n_rhs, const int* skip, cudaStream_t s, cudaEvent_t* ev = nullptr, int reps = 1,
                         const TileSet* ts = nullptr, int skip_stride = 0);

// Deterministic plans: the operator writes its weighted timestream (no
// scatter), then k_segsum adds each row's samples in ascending order.
template <typename Real, int NS, int IN>
madmap_status launch_det(Plan* p, const void* in, void* out, long long in_stride, long long out_stride, int n_rhs,
                         const int* skip, cudaStream_t s, cudaEvent_t* ev, int reps, const TileSet* ts,
                         int skip_stride) {
  typedef typename OutT<Real>::type Out;
  constexpr int NSI = gathers(IN) ? NS : 1;   // a timestream input needs no pointing
  const int nr = ts ? ts->n_rhs : 1;
  MM_CHECK(p->wtod && p->wtod_rhs >= nr, MADMAP_ERR_INTERNAL, "deterministic plan without a timestream buffer");
  const int grid_x = (int)std::max(1LL, std::min<long long>(((long long)p->n_obs + 7) / 8, 152LL * 16));
  if (n_rhs == 0) return launch_all<Real, NSI, IN, OUT_TOD>(p, in, p->wtod, 0, 0, 0, skip, s, nullptr, 1, ts, 0);
  for (int rep = 0; rep < reps; ++rep) {
    if (ts) {
      madmap_status st = launch_all<Real, NSI, IN, OUT_TOD>(p, in, p->wtod, in_stride, p->n_t, 1, skip, s, ev, 1,
                                                            ts, skip_stride);
      if (st != MADMAP_OK) return st;
      k_segsum<Real, NS><<<dim3(grid_x, nr), 256, 0, s>>>(static_cast<const Out*>(p->wtod), p->n_t, p->det_ptr,
                                                         p->det_idx, p->n_obs, p->psi, p->cs64,
                                                         static_cast<Out*>(out), out_stride, skip, skip_stride);
      count_launches(1);
      continue;
    }
    for (int r = 0; r < n_rhs; ++r) {
      const void* in_r = static_cast<const char*>(in) + (size_t)r * in_stride *
                                                            (IN == IN_TODF ? sizeof(float) : sizeof(Real));
      Out* out_r = static_cast<Out*>(out) + (size_t)r * out_stride;
      madmap_status st = launch_all<Real, NSI, IN, OUT_TOD>(p, in_r, p->wtod, 0, 0, 1, skip, s, ev, 1, nullptr, 0);
      if (st != MADMAP_OK) return st;
      k_segsum<Real, NS><<<dim3(grid_x, 1), 256, 0, s>>>(static_cast<const Out*>(p->wtod), 0, p->det_ptr,
                                                        p->det_idx, p->n_obs, p->psi, p->cs64, out_r, 0, skip, 0);
      count_launches(1);
    }
  }
  MM_CUDA(cudaGetLastError());
  return MADMAP_OK;
}

template <typename Real, int NS, int IN, int OUT>
madmap_status launch_all(Plan* p, const void* in, void* out, long long in_stride, long long out_stride,
                         int n_rhs, const int* skip, cudaStream_t s, cudaEvent_t* ev, int reps,
                         const TileSet* ts, int skip_stride) {
  if constexpr (OUT == OUT_MAP && (NS == 1 || NS == 3)) {
    if (p->det) return launch_det<Real, NS, IN>(p, in, out, in_stride, out_stride, n_rhs, skip, s, ev, reps, ts,
                                                skip_stride);
  }
  OpArgs a;
  a.M = p->M;
  a.N1 = p->N1;
  a.N2 = p->N2;
  a.logN1 = p->logN1;
  a.logN2 = p->logN2;
  geometry<Real>(p, a.B1, a.B2);
  a.logB1 = ilog2((unsigned)a.B1);
  a.pix = p->pix_obs;
  a.psi = p->psi;
  a.cs64 = p->cs64;
  a.csdf = p->csdf;
  a.pw = p->pw;
  a.pixq = p->pix_obs_pol;
  a.ext = p->ext_row;
  a.hwp_base = p->hwp_base;
  a.hwp_ang = p->hwp_ang;
  a.hwp_tau = p->hwp_tau;
  a.bore = p->otf ? p->bore : nullptr;
  a.det = p->det_pt;
  a.g2o = p->g2o;
  a.sd = make_step_div(p->bore_step > 0 ? p->bore_step : 1);
  a.n_per_det = p->n_per_det;
  a.n_det = p->n_det;
  a.grid_w = p->grid_w;
  a.grid_h = p->grid_h;
  a.scratch = p->scratch;
  constexpr bool DF = std::is_same<Real, df64>::value;
  a.H = DF ? (const void*)p->Hdf : sizeof(Real) == 8 ? (const void*)p->H64 : (const void*)p->H32;
  a.tw = DF ? (const void*)p->twdf : sizeof(Real) == 8 ? (const void*)p->tw64 : (const void*)p->tw32;
  a.skip = skip;
  a.skip_stride = ts ? skip_stride : 0;
  a.in2 = p->resid_d;
  a.in2_stride = p->resid_stride;
  a.n_rep = 1;
  a.rep_stride = 0;
  a.runs = p->runs;
  a.tiles = ts ? ts->tiles : p->tiles;
  const int n_tiles = ts ? ts->n_tiles : p->n_tiles;
  const size_t sm13 = smem_f13<Real>(p), sm2 = smem_f2<Real>(p);
  const OpKernels K = pick_kernels<Real, NS, IN, OUT>(p);
  // n_rhs == 0 only sets the kernels' attributes, so it can precede a capture
  MM_CUDA(set_smem(K.f1, sm13));
  MM_CUDA(set_smem(K.f3, sm13));
  MM_CUDA(set_smem(K.f2, sm2));
  if (p->diag && !ts) {
    // white noise: one diagonal pass per right-hand side (launch events as
    // four per application so per-kernel timing keeps its layout)
    for (int rep = 0; rep < reps; ++rep)
      for (int r = 0; r < n_rhs; ++r) {
        a.in = static_cast<const char*>(in) + (size_t)r * in_stride * (IN == IN_TODF ? sizeof(float) : sizeof(Real));
        a.out = static_cast<char*>(out) + (size_t)r * out_stride * sizeof(typename OutT<Real>::type);
        a.in_stride = a.out_stride = 0;
        if (IN == IN_RESX) a.in2 = p->resid_d + (size_t)r * p->resid_stride;
        if (ev) cudaEventRecord(ev[4 * (rep * n_rhs + r)], s);
        if constexpr (extended(NS) && OUT == OUT_MAP) {
          if (p->hwp_base)
            k_diag<Real, NS, IN, OUT, true><<<p->n_diag_items, 256, 0, s>>>(a, p->diag_items, p->f0_64);
          else
            k_diag<Real, NS, IN, OUT, false><<<p->n_diag_items, 256, 0, s>>>(a, p->diag_items, p->f0_64);
        } else {
          k_diag<Real, NS, IN, OUT, false><<<p->n_diag_items, 256, 0, s>>>(a, p->diag_items, p->f0_64);
        }
        if (ev)
          for (int k = 1; k < 4; ++k) cudaEventRecord(ev[4 * (rep * n_rhs + r) + k], s);
      }
    count_launches((long long)n_rhs * reps);
    MM_CUDA(cudaGetLastError());
    return MADMAP_OK;
  }
  int n_chunks, per_chunk;
  chunking(p, n_chunks, per_chunk, n_tiles);
  // map replicas for small, heavily hit maps (single right-hand side per launch)
  typedef typename OutT<Real>::type Out;
  const bool use_rep = !ts && OUT == OUT_MAP && p->n_rep > 1 && p->rep;
  const long long n_map = (long long)std::max(1, p->n_obs) * p->ns_pad;
  // several chunks: alternate two streams (own scratch slot each) so chunks overlap
  // (with replicas only when one application is enqueued: the replicas are reused)
  const bool pipe = !ev && n_rhs > 0 && n_chunks > 1 && p->op_stream[0] && p->scratch_slots > 1 &&
                    (!use_rep || n_rhs * reps == 1);
  const int rgrid = (int)std::min<long long>((n_map + 255) / 256, 152LL * 8);
  const size_t slot_bytes = (size_t)p->tiles_per_chunk * p->M * sizeof(double2);
  if (pipe) {
    MM_CUDA(cudaEventRecord(p->op_fork, s));
    for (int i = 0; i < 2; ++i) MM_CUDA(cudaStreamWaitEvent(p->op_stream[i], p->op_fork, 0));
  }
  int ei = 0, chunk = 0;
  for (int rep = 0; rep < reps; ++rep) {
    for (int r = 0; r < n_rhs; ++r) {
      a.in = static_cast<const char*>(in) + (size_t)r * in_stride *
                                                (IN == IN_TODF ? sizeof(float) : sizeof(Real));
      if (IN == IN_RESX && !ts) a.in2 = p->resid_d + (size_t)r * p->resid_stride;
      a.out = static_cast<char*>(out) + (size_t)r * out_stride * sizeof(typename OutT<Real>::type);
      Out* const map_out = static_cast<Out*>(a.out);
      if (use_rep) {
        a.out = p->rep;
        a.n_rep = p->n_rep;
        a.rep_stride = n_map;
      }
      // a tile set names each lane's right-hand side, with per-rhs strides;
      // otherwise the plan's tiles are replayed once per right-hand side
      a.in_stride = ts ? in_stride : 0;
      a.out_stride = ts ? out_stride : 0;
      for (int t0 = 0; t0 < n_tiles; t0 += per_chunk) {
        const int nt = (n_tiles - t0) < per_chunk ? (n_tiles - t0) : per_chunk;
        a.tile0 = t0;
        const cudaStream_t cs = pipe ? p->op_stream[chunk & 1] : s;
        a.scratch = static_cast<char*>(p->scratch) + (pipe ? (size_t)(chunk & 1) * slot_bytes : 0);
        ++chunk;
        dim3 g13(p->N1 / a.B1, nt), g2(p->N2 / a.B2, nt);
        if (ev) cudaEventRecord(ev[ei++], s);
        K.f1<<<g13, OP_THREADS, sm13, cs>>>(a);
        if (ev) cudaEventRecord(ev[ei++], s);
        K.f2<<<g2, OP_THREADS, sm2, cs>>>(a);
        if (ev) cudaEventRecord(ev[ei++], s);
        K.f3<<<g13, OP_THREADS, sm13, cs>>>(a);
        if (ev) cudaEventRecord(ev[ei++], s);
      }
      if (use_rep) {
        if (pipe) {
          for (int i = 0; i < 2; ++i) {
            MM_CUDA(cudaEventRecord(p->op_join[i], p->op_stream[i]));
            MM_CUDA(cudaStreamWaitEvent(s, p->op_join[i], 0));
          }
        }
        k_rep_reduce<Out><<<rgrid, 256, 0, s>>>(static_cast<Out*>(p->rep), p->n_rep, n_map, map_out, n_map);
        count_launches(1);
      }
    }
  }
  if (pipe && !use_rep) {
    for (int i = 0; i < 2; ++i) {
      MM_CUDA(cudaEventRecord(p->op_join[i], p->op_stream[i]));
      MM_CUDA(cudaStreamWaitEvent(s, p->op_join[i], 0));
    }
  }
  count_launches(3LL * n_chunks * n_rhs * reps);
  MM_CUDA(cudaGetLastError());
  return MADMAP_OK;
}

template <typename Real, int NS>
madmap_status dispatch_io(Plan* p, int in_mode, int out_mode, const void* in, void* out, long long is,
                          long long os, int n_rhs, const int* skip, cudaStream_t s) {
  if (in_mode == IN_MAP && out_mode == OUT_MAP)
    return launch_all<Real, NS, IN_MAPX, OUT_MAP>(p, in, out, is, os, n_rhs, skip, s);
  if (in_mode == IN_TOD && out_mode == OUT_MAP)
    return launch_all<Real, NS, IN_TODF, OUT_MAP>(p, in, out, is, os, n_rhs, skip, s);
  if (in_mode == IN_TOD_REAL && out_mode == OUT_TOD)  // no pointing: the T instance serves every layout
    return launch_all<Real, 1, IN_TODR, OUT_TOD>(p, in, out, is, os, n_rhs, skip, s);
  if (in_mode == IN_MAP && out_mode == OUT_TOD)
    return launch_all<Real, NS, IN_MAPX, OUT_TOD>(p, in, out, is, os, n_rhs, skip, s);
  if constexpr ((NS == 1 || NS == 3) && !std::is_same<Real, float>::value) {
    if (in_mode == IN_RESID && out_mode == OUT_MAP)
      return launch_all<Real, NS, IN_RESX, OUT_MAP>(p, in, out, is, os, n_rhs, skip, s);
  }
  set_error("unsupported operator mode");
  return MADMAP_ERR_INTERNAL;
}

// double-float: map or float timestream in, float64 map out
template <int NS>
madmap_status dispatch_df(Plan* p, int in_mode, int out_mode, const void* in, void* out, long long is, long long os,
                          int n_rhs, const int* skip, cudaStream_t s) {
  if (in_mode == IN_MAP && out_mode == OUT_MAP)
    return launch_all<df64, NS, IN_MAPX, OUT_MAP>(p, in, out, is, os, n_rhs, skip, s);
  if (in_mode == IN_TOD && out_mode == OUT_MAP)
    return launch_all<df64, NS, IN_TODF, OUT_MAP>(p, in, out, is, os, n_rhs, skip, s);
  if constexpr (NS == 1 || NS == 3) {
    if (in_mode == IN_RESID && out_mode == OUT_MAP)
      return launch_all<df64, NS, IN_RESX, OUT_MAP>(p, in, out, is, os, n_rhs, skip, s);
  }
  set_error("unsupported double-float operator mode");
  return MADMAP_ERR_INTERNAL;
}

template <typename Real, int NS>
madmap_status time_impl(Plan* p, const void* in, void* out, int reps, double ms[4], cudaStream_t s) {
  int n_chunks, per_chunk;
  chunking(p, n_chunks, per_chunk);
  const int n_ev = reps * n_chunks * 4;
  std::vector<cudaEvent_t> ev(n_ev, nullptr);
  madmap_status st = MADMAP_OK;
  for (int i = 0; i < n_ev && st == MADMAP_OK; ++i)
    if (cudaEventCreate(&ev[i]) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "cudaEventCreate");
  if (st == MADMAP_OK) {
    const long long nv = (long long)std::max(1, p->n_obs) * p->ns_pad;
    for (int rep = 0; rep < reps && st == MADMAP_OK; ++rep) {
      if (cudaMemsetAsync(out, 0, sizeof(typename OutT<Real>::type) * nv, s) != cudaSuccess)
        st = cuda_fail(cudaGetLastError(), "memset");
      if (st == MADMAP_OK)
        st = launch_all<Real, NS, IN_MAPX, OUT_MAP>(p, in, out, 0, 0, 1, nullptr, s, ev.data() + rep * n_chunks * 4, 1);
    }
  }
  if (st == MADMAP_OK && cudaStreamSynchronize(s) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "sync");
  // whole applications as the solver launches them (chunks overlapped)
  cudaEvent_t a0 = nullptr, a1 = nullptr;
  if (st == MADMAP_OK && (cudaEventCreate(&a0) != cudaSuccess || cudaEventCreate(&a1) != cudaSuccess))
    st = cuda_fail(cudaGetLastError(), "cudaEventCreate");
  if (st == MADMAP_OK) {
    const long long nv = (long long)std::max(1, p->n_obs) * p->ns_pad;
    cudaEventRecord(a0, s);
    for (int rep = 0; rep < reps && st == MADMAP_OK; ++rep) {
      if (cudaMemsetAsync(out, 0, sizeof(typename OutT<Real>::type) * nv, s) != cudaSuccess)
        st = cuda_fail(cudaGetLastError(), "memset");
      if (st == MADMAP_OK) st = launch_all<Real, NS, IN_MAPX, OUT_MAP>(p, in, out, 0, 0, 1, nullptr, s);
    }
    cudaEventRecord(a1, s);
    if (st == MADMAP_OK && cudaStreamSynchronize(s) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "sync");
    float t = 0.f;
    if (st == MADMAP_OK) cudaEventElapsedTime(&t, a0, a1);
    ms[3] = t / reps;
  }
  if (a0) cudaEventDestroy(a0);
  if (a1) cudaEventDestroy(a1);
  if (st == MADMAP_OK) {
    ms[0] = ms[1] = ms[2] = 0.0;
    for (int c = 0; c < reps * n_chunks; ++c)
      for (int k = 0; k < 3; ++k) {
        float t = 0.f;
        cudaEventElapsedTime(&t, ev[c * 4 + k], ev[c * 4 + k + 1]);
        ms[k] += t;
      }
    for (int k = 0; k < 3; ++k) ms[k] /= (double)(reps * n_chunks);
  }
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  return st;
}

template <typename Real, int NS>
madmap_status dispatch_set(Plan* p, int in_mode, int out_mode, const void* in, void* out, long long is,
                           long long os, const int* skip, int ss, cudaStream_t s, const TileSet* ts) {
  if (in_mode == IN_MAP && out_mode == OUT_MAP)
    return launch_all<Real, NS, IN_MAPX, OUT_MAP>(p, in, out, is, os, 1, skip, s, nullptr, 1, ts, ss);
  if (in_mode == IN_TOD && out_mode == OUT_MAP)
    return launch_all<Real, NS, IN_TODF, OUT_MAP>(p, in, out, is, os, 1, skip, s, nullptr, 1, ts, ss);
  if constexpr ((NS == 1 || NS == 3) && !std::is_same<Real, float>::value) {
    if (in_mode == IN_RESID && out_mode == OUT_MAP)
      return launch_all<Real, NS, IN_RESX, OUT_MAP>(p, in, out, is, os, 1, skip, s, nullptr, 1, ts, ss);
  }
  set_error("unsupported batched operator mode");
  return MADMAP_ERR_INTERNAL;
}

// ---------------------------------------------------------------- per-precision entry points
// Each precision's kernels are compiled in a translation unit of their own
// (operator_f32.cu, operator_f64.cu, operator_df64.cu), which exports an
// OpImpl table built from these templates.
template <typename Real>
madmap_status impl_launch(Plan* p, int in_mode, int out_mode, const void* in, void* out, long long is,
                          long long os, int n_rhs, const int* skip, cudaStream_t s) {
  const int k = layout(p);
  if constexpr (std::is_same<Real, df64>::value) {
#define MM_DF(NSV) dispatch_df<NSV>(p, in_mode, out_mode, in, out, is, os, n_rhs, skip, s)
    return MM_FOR_LAYOUT(k, MM_DF);
#undef MM_DF
  } else {
#define MM_IO(NSV) dispatch_io<Real, NSV>(p, in_mode, out_mode, in, out, is, os, n_rhs, skip, s)
    return MM_FOR_LAYOUT(k, MM_IO);
#undef MM_IO
  }
}

template <typename Real>
madmap_status impl_launch_set(Plan* p, int in_mode, int out_mode, const void* in, void* out, long long is,
                              long long os, const int* skip, int ss, const TileSet* ts, cudaStream_t s) {
  const int k = layout(p);
#define MM_SET(NSV) dispatch_set<Real, NSV>(p, in_mode, out_mode, in, out, is, os, skip, ss, s, ts)
  return MM_FOR_LAYOUT(k, MM_SET);
#undef MM_SET
}

template <typename Real>
madmap_status impl_time(Plan* p, const void* in, void* out, int reps, double ms[4], cudaStream_t s) {
  const int k = layout(p);
#define MM_TIME(NSV) time_impl<Real, NSV>(p, in, out, reps, ms, s)
  return MM_FOR_LAYOUT(k, MM_TIME);
#undef MM_TIME
}

// Resident CTAs per SM of the map-to-map kernels (the least of the three) and
// CTAs per tile of the column kernels, for wave-aligned chunk sizes.
template <typename Real>
void impl_occupancy(const Plan* p, int& ctas_per_sm, int& ctas_per_tile) {
  int b1 = 0, b2 = 0, n1 = 0, n2 = 0, n3 = 0;
  geometry<Real>(p, b1, b2);
  const size_t s13 = smem_f13<Real>(p), s2 = smem_f2<Real>(p);
  const int k = layout(p);
#define MM_PICK(NSV) pick_kernels<Real, NSV, IN_MAPX, OUT_MAP>(p)
  const OpKernels K = MM_FOR_LAYOUT(k, MM_PICK);
#undef MM_PICK
  set_smem(K.f1, s13);
  set_smem(K.f2, s2);
  set_smem(K.f3, s13);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n1, K.f1, OP_THREADS, s13);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n2, K.f2, OP_THREADS, s2);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n3, K.f3, OP_THREADS, s13);
  cudaGetLastError();
  ctas_per_sm = std::max(1, std::min(n1, std::min(n2, n3)));
  ctas_per_tile = std::max(1, p->N1 / std::max(1, b1));
}

template <typename Real>
size_t impl_f13_smem(const Plan* p) {
  return smem_f13<Real>(p);
}

template <typename Real>
madmap_status impl_weights(long long n, const float* psi, void* c, void* s, cudaStream_t st) {
  if constexpr (std::is_same<Real, df64>::value) {
    set_error("weights: no double-float instance");
    return MADMAP_ERR_INTERNAL;
  } else {
    if (n <= 0) return MADMAP_OK;
    const int grid = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    k_weights<Real><<<grid, 256, 0, st>>>(n, psi, static_cast<Real*>(c), static_cast<Real*>(s));
    count_launches(1);
    MM_CUDA(cudaGetLastError());
    return MADMAP_OK;
  }
}

template <typename Real>
OpImpl make_impl() {
  OpImpl t;
  t.weights = impl_weights<Real>;
  t.launch = impl_launch<Real>;
  t.launch_set = impl_launch_set<Real>;
  t.time = impl_time<Real>;
  if constexpr (std::is_same<Real, df64>::value) t.occupancy = nullptr;
  else t.occupancy = impl_occupancy<Real>;
  t.f13_smem = impl_f13_smem<Real>;
  return t;
}

}  // namespace
}  // namespace mm
