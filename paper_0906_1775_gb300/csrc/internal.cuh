// Internal declarations of libmadmap: plan layout, device helpers and the
// shared-memory radix FFT used by the noise-weighting kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "madmap.h"

namespace mm {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
madmap_status cuda_fail(cudaError_t e, const char* what);

#define MM_CUDA(call)                                             \
  do {                                                            \
    cudaError_t e__ = (call);                                     \
    if (e__ != cudaSuccess) return ::mm::cuda_fail(e__, #call);   \
  } while (0)

#define MM_CHECK(cond, status, msg)       \
  do {                                    \
    if (!(cond)) {                        \
      ::mm::set_error(msg);               \
      return (status);                    \
    }                                     \
  } while (0)

// ---------------------------------------------------------------- geometry
// One real overlap-save window (a "lane"): complex-FFT position n of the
// window holds sample t = ws + n when lo <= t < hi (else zero); outputs are
// kept for window positions out_lo <= n < out_hi.
struct Lane {
  long long ws, lo, hi;
  int out_lo, out_hi, rhs, pad;
};
// Two lanes share one complex FFT (lane 0 in the real part, lane 1 in the
// imaginary part).  Both use the same filter: its circulant spectrum is real
// and even, so the product keeps the two real lanes apart.
struct Tile {
  Lane l[2];
  int filter;
  int pad[3];
};

// White noise (one filter lag): a run of samples of one interval, weighted by
// its filter's f(0) in a single pass (no windows, no FFT).
struct DiagItem {
  long long lo, hi;
  int filter, pad;
};

// A list of tiles whose lanes name their right-hand side (batched solves).
struct TileSet {
  Tile* tiles = nullptr;  // device
  int n_tiles = 0;
  int n_rhs = 0;
};

// ---------------------------------------------------------------- double-float
// A double-float number is the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi) / 2: about 48 significant bits from float32 arithmetic.
// Sums use Knuth's two-sum for the high parts, products Dekker's exact
// product through a fused multiply-add; the error terms are folded in once
// and renormalised (the double-double scheme of Hida, Li and Bailey, 2001,
// at float width).  The intrinsics keep the compiler from contracting the
// error-free steps.  On GB300 these run at the float32 rate, far above the
// float64 rate.
struct __align__(8) df64 {
  float hi, lo;
  __host__ __device__ constexpr df64() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr df64(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ constexpr df64(float v) : hi(v), lo(0.f) {}
  __host__ __device__ constexpr df64(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
};
struct __align__(16) cdf64 {
  df64 x, y;
};
__host__ __device__ inline double to_double(df64 a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ df64 df_renorm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return df64(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_renorm(s, e);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_renorm(p, e);
}
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }

// ---------------------------------------------------------------- compressed pointing
// Division of a detector sample index j >= 0 by the node step: a shift for a
// power of two, else a multiply-high by a precomputed reciprocal (division by
// invariant integers, Granlund and Montgomery, PLDI 1994) followed by one
// correction step, so the quotient is exact for every j < 2^31.
struct StepDiv {
  int step = 1, shift = 0;   // shift: log2(step) (power of two) or ceil(log2(step)) - 1
  unsigned magic = 0;        // 0 for a power of two
  float inv = 1.f;           // 1 / step (exact for a power of two)
};
inline StepDiv make_step_div(int step) {
  StepDiv d;
  d.step = step;
  int l = 0;
  while ((1LL << l) < step) ++l;
  if ((1LL << l) == step) {
    d.shift = l;
    d.magic = 0;
    d.inv = 1.0f / (float)step;
  } else {
    // m = ceil(2^(31 + l) / step) < 2^32
    const unsigned long long num = 1ULL << (31 + l);
    d.magic = (unsigned)((num + (unsigned long long)step - 1) / (unsigned long long)step);
    d.shift = l - 1;
    d.inv = 0.f;
  }
  return d;
}
__device__ __forceinline__ int step_quot(const StepDiv& d, int j, int& r) {
  int q;
  if (d.magic == 0) {
    q = j >> d.shift;
  } else {
    q = (int)(__umulhi((unsigned)j, d.magic) >> d.shift);
    const int rr = j - q * d.step;
    if (rr < 0) --q;
    else if (rr >= d.step) ++q;
  }
  r = j - q * d.step;
  return q;
}

// Section 5.3: the pointing of detector sample j (detector pointing dp =
// (dx, dy, cd, sd)) expanded from the boresight nodes, in the float32
// operation order stated with madmap_plan_desc (no contraction, so the pixel
// decisions are reproducible).  Returns the global pixel or -1; c2, s2 get
// cos 2psi and sin 2psi when `pol`.  FAST_W: the weights' two divisions by n
// become one approximate reciprocal (relative error ~1e-7, for the float32
// operator); the pixel decision is the same either way.
template <bool FAST_W = false>
__device__ __forceinline__ int expand_pointing(const float4* __restrict__ bore, const StepDiv& sd, int j, float4 dp,
                                               int W, int H, bool pol, float& c2, float& s2) {
  int r;
  const int u = step_quot(sd, j, r);
  const float f = sd.magic == 0 ? __fmul_rn((float)r, sd.inv) : __fdiv_rn((float)r, (float)sd.step);
  const float4 a = __ldg(bore + u), b = __ldg(bore + u + 1);
  const float x = __fadd_rn(a.x, __fmul_rn(f, __fsub_rn(b.x, a.x)));
  const float y = __fadd_rn(a.y, __fmul_rn(f, __fsub_rn(b.y, a.y)));
  const float c = __fadd_rn(a.z, __fmul_rn(f, __fsub_rn(b.z, a.z)));
  const float s = __fadd_rn(a.w, __fmul_rn(f, __fsub_rn(b.w, a.w)));
  const float X = __fadd_rn(x, __fsub_rn(__fmul_rn(c, dp.x), __fmul_rn(s, dp.y)));
  const float Y = __fadd_rn(y, __fadd_rn(__fmul_rn(s, dp.x), __fmul_rn(c, dp.y)));
  const float fx = floorf(X), fy = floorf(Y);
  bool ok = fx >= 0.f && fx < (float)W && fy >= 0.f && fy < (float)H;
  c2 = s2 = 0.f;
  if (pol) {
    const float C = __fsub_rn(__fmul_rn(c, dp.z), __fmul_rn(s, dp.w));
    const float S = __fadd_rn(__fmul_rn(s, dp.z), __fmul_rn(c, dp.w));
    const float cc = __fmul_rn(C, C), ss = __fmul_rn(S, S);
    const float n = __fadd_rn(cc, ss);
    const float cs = __fmul_rn(C, S);
    ok = ok && n > 0.f;
    if (ok) {
      if (FAST_W) {
        const float in = __fdividef(1.0f, n);
        c2 = (cc - ss) * in;
        s2 = (cs + cs) * in;
      } else {
        c2 = __fdiv_rn(__fsub_rn(cc, ss), n);
        s2 = __fdiv_rn(__fadd_rn(cs, cs), n);
      }
    }
  }
  return ok ? (int)fy * W + (int)fx : -1;
}

// base[idx] += v for the calling lanes with one atomic per distinct idx in the
// warp: lanes that share an address (an extra column of extended pointing is
// shared by a whole baseline of consecutive samples, a half-wave-plate
// parameter by a whole interval) add up their values by shuffles first, so no
// address takes a stream of atomics from one warp.
template <typename Out>
__device__ __forceinline__ void atomic_add_warp(Out* base, long long idx, Out v) {
  const unsigned active = __activemask();
  const unsigned peers = __match_any_sync(active, (unsigned long long)idx);
  Out acc = Out(0);
  if (peers == 0xffffffffu) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(peers, v, o);
    acc = v;
  } else {
    for (unsigned m = peers; m; m &= m - 1) acc += __shfl_sync(peers, v, __ffs(m) - 1);
  }
  if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(base + idx, acc);
}

// Half-wave-plate columns of one sample (Section 6, Eq. 42), in the column
// order b_1..b_32: cos k w, tau cos k w, sin k w, tau sin k w for k = 1..8.
// The harmonics come from one sincos by the angle-addition recurrence.
template <typename W>
__device__ __forceinline__ void hwp_columns(float w, float tau, W* C) {
  W c1, s1;
  if constexpr (sizeof(W) == 4) sincosf(w, &s1, &c1);
  else sincos((double)w, &s1, &c1);
  W c = c1, s = s1;
  const W t = (W)tau;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    C[k] = c;
    C[8 + k] = t * c;
    C[16 + k] = s;
    C[24 + k] = t * s;
    const W cn = c * c1 - s * s1;
    s = s * c1 + c * s1;
    c = cn;
  }
}

// The compressed pointing of a plan as kernel arguments (bore == NULL: the
// plan stores per-sample pointing instead).
struct OtfPointing {
  const float4* bore;
  const float4* det;
  const int* g2o;
  StepDiv sd;
  int n_per_det, W, H;
};

// Observed row of sample t (or -1) and its weights, from compressed pointing.
__device__ __forceinline__ int otf_row(const OtfPointing& o, long long t, bool pol, float& c2, float& s2) {
  const int dd = (int)(t / o.n_per_det);
  const int g = expand_pointing(o.bore, o.sd, (int)(t - (long long)dd * o.n_per_det), o.det[dd], o.W, o.H, pol, c2,
                                s2);
  return g >= 0 ? o.g2o[g] : -1;
}

// ---------------------------------------------------------------- plan
struct SolveBuffers;  // solver.cu

struct Plan {
  // description
  int n_stokes = 1, ns_pad = 1;
  long long n_t = 0;
  int n_pix = 0, n_obs = 0, n_excised = 0, n_fp64 = 0;
  int n_ivl = 0, n_filters = 0, n_lags = 0;
  double rcond_excise = 1e-6, rcond_fp64 = 1e-2;
  std::vector<long long> offsets;
  std::vector<int> ivl_filter;
  std::vector<double> lags;
  // FFT geometry: M = N1 * N2; F1/F3 handle B1 columns per CTA, F2 handles B2 rows
  int M = 0, N1 = 0, N2 = 0, logN1 = 0, logN2 = 0;
  int n_segments = 0, n_tiles = 0, tiles_per_chunk = 0;
  std::vector<Tile> host_tiles;
  // device buffers owned by the plan
  int* pix_obs = nullptr;          // [n_t] observed pixel or -1
  float* psi = nullptr;            // [n_t] copy of the angles (IQU)
  double2* cs64 = nullptr;         // [n_t] (cos 2psi, sin 2psi) in float64 (IQU)
  int* obs2glob = nullptr;         // [n_obs]
  unsigned char* excised = nullptr;   // [n_obs]
  unsigned char* fp64flag = nullptr;  // [n_obs]
  double* P64 = nullptr;           // [n_obs][6] (IQU) or [n_obs] (T): block inverses
  float* P32 = nullptr;            // [n_obs][8] (IQU) or [n_obs] (T)
  Tile* tiles = nullptr;           // [n_tiles]
  double* H64 = nullptr;           // [n_filters][M] permuted spectra / M
  float* H32 = nullptr;
  double2* tw64 = nullptr;         // [M] exp(-2 pi i j / M)
  float2* tw32 = nullptr;
  df64* Hdf = nullptr;             // [n_filters][M] H64 as double-float pairs
  cdf64* twdf = nullptr;           // [M] tw64 as double-float pairs
  float4* csdf = nullptr;          // [n_t] cs64 as double-float pairs (IQU)
  int2* pw = nullptr;              // [n_t] (pix_obs, bits of psi) for the float32 operator (IQU)
  int* hits = nullptr;             // [n_obs] samples per pixel before excision
  double* G = nullptr;             // [n_filters][n_obs][6] (IQU) or [n_filters][n_obs] (T): sums of w w^T
                                   // per filter, kept when they fit 512 MB (fast filter changes)
  bool pre_built = false;          // the preconditioner has been built once
  // multi-resolution maps: Q/U on a second pixelisation; vectors are slots
  // holding I of I pixel k and Q, U of Q/U pixel k (n_obs = max of the counts)
  bool multires = false;
  int n_pix_pol = 0, n_obs_i = 0, n_obs_pol = 0, n_excised_pol = 0;
  int* pix_obs_pol = nullptr;      // [n_t] observed Q/U pixel or -1
  int* obs2glob_pol = nullptr;     // [n_obs_pol]
  unsigned char* excised_pol = nullptr;  // [n_obs] (slots)
  // pointing expanded on the fly from compressed boresight pointing (no
  // per-sample arrays: pix_obs, psi, cs64, csdf, pw stay NULL)
  bool otf = false;
  const float4* bore = nullptr;    // [n_bore] device copy of the nodes
  float4* det_pt = nullptr;        // [n_det] detector offsets and orientations
  int n_bore = 0, bore_step = 1, n_det = 0, n_per_det = 0, grid_w = 0, grid_h = 0;
  int* g2o = nullptr;              // [n_pix] observed row of each global pixel, -1 if unobserved or excised
  // extended pointing: extra unit-weight columns after the sky rows
  bool ext = false;
  int n_extra = 0, n_obs_sky = 0, n_excised_extra = 0;
  int* ext_row = nullptr;          // [n_t] map row of the sample's extra column (n_obs_sky + e) or -1
  // half-wave-plate parameters (32 rows per group after the extra rows)
  int n_hwp_groups = 0, hwp_row0 = 0, n_excised_hwp = 0;
  float* hwp_ang = nullptr;        // [n_t] polariser angle
  float* hwp_tau = nullptr;        // [n_t] the model's time variable
  int* hwp_base = nullptr;         // [n_t] first row of the sample's group, or -1
  // small maps hit by many samples: the operator's scatter spreads over n_rep
  // replicas of the map (picked per CTA) that one kernel then adds up, so no
  // address takes every sample's atomic
  int n_rep = 1;
  void* rep = nullptr;             // n_rep x n_obs x ns_pad (float64 size), zero between applications
  // samples whose successor hits the same observed pixel (a measure of how
  // slowly the scan crosses pixels), and whether the column kernels' scatter
  // sums such runs of lanes before one atomic per run
  double repeat_frac = 0.0;
  int runs = 0;
  bool runs_fixed = false;         // set by the description, not by the autotuner
  // white noise (n_lags == 1): the operator is one diagonal pass over sample runs
  bool diag = false;
  DiagItem* diag_items = nullptr;  // [n_diag_items]
  int n_diag_items = 0;
  double* f0_64 = nullptr;         // [n_filters] f(0) of each filter
  void* scratch = nullptr;         // scratch_slots * tiles_per_chunk * M complex (float64 size)
  int scratch_slots = 1;           // 2 when an application has several chunks (see op_stream)
  // An application of several chunks alternates them between two streams,
  // each with its own scratch slot, so one chunk's kernels overlap the
  // previous chunk's tail and its scratch and pointing stay in L2.
  cudaStream_t op_stream[2] = {nullptr, nullptr};
  cudaEvent_t op_fork = nullptr;
  cudaEvent_t op_join[2] = {nullptr, nullptr};
  int* dev_flag = nullptr;         // small device flag words
  size_t device_bytes = 0;
  std::vector<void*> allocs;
  SolveBuffers* sb64 = nullptr;
  SolveBuffers* sb32 = nullptr;
  // solves run on a plan-owned non-blocking stream (graph capture is not
  // allowed on the legacy default stream), ordered after the caller's stream
  cudaStream_t solve_stream = nullptr;
  cudaEvent_t solve_event = nullptr;
  std::vector<TileSet*> tile_sets;  // batched tile lists by n_rhs (device memory in allocs)
  // backward pass: timestreams A lambda and d - A m, lag-correlation work items
  float* bw_a = nullptr;
  float* bw_r = nullptr;
  void* corr_items = nullptr;
  int n_corr_items = 0;
  // deterministic plans: the samples of every observed row in ascending order
  // (rows det_ptr[p] .. det_ptr[p+1]-1 of det_idx), and the timestream buffer
  // the operator writes before the ordered row sums ([wtod_rhs][n_t], float64 size)
  bool det = false;
  int* det_ptr = nullptr;
  int* det_idx = nullptr;
  void* wtod = nullptr;
  int wtod_rhs = 0;
  // buffers that depend on the FFT length (freed and rebuilt by the autotuner)
  std::vector<void*> win_allocs;
  size_t win_bytes = 0;
  // the autotuner's candidates: FFT length, tiles per chunk, float32 operator ms
  struct Tuned {
    int M, tpc;
    float ms;
    int runs, n2;
  };
  int split_down = 0;              // column transforms of 2^(ceil(log2 M / 2) - split_down) points
  bool split_fixed = false;        // set by the description, not by the autotuner
  std::vector<Tuned> tuned;
  // the data timestream of an IN_RESID operator application (set by the
  // caller around the launch)
  const float* resid_d = nullptr;
  long long resid_stride = 0;
  // sharded solves: sums map-domain buffers across the ranks (NULL: one process)
  madmap_reduce_fn allreduce = nullptr;
  void* allreduce_user = nullptr;
  ~Plan();
};

// Sums a device buffer across the ranks of a sharded plan (nothing to do for
// a single-process plan).  dtype: MADMAP_REDUCE_F64 / F32 / I32.
madmap_status reduce_across(Plan* p, void* buf, long long count, int dtype, cudaStream_t s);

inline OtfPointing otf_pointing(const Plan* p) {
  OtfPointing a;
  a.bore = p->otf ? p->bore : nullptr;
  a.det = p->det_pt;
  a.g2o = p->g2o;
  a.sd = make_step_div(p->bore_step > 0 ? p->bore_step : 1);
  a.n_per_det = p->n_per_det > 0 ? p->n_per_det : 1;
  a.W = p->grid_w;
  a.H = p->grid_h;
  return a;
}

madmap_status dalloc(Plan* p, void** ptr, size_t bytes);
template <typename T>
inline madmap_status dalloc_t(Plan* p, T** ptr, size_t count) {
  return dalloc(p, reinterpret_cast<void**>(ptr), count * sizeof(T));
}

// ---------------------------------------------------------------- operator launch
// Arithmetic of an operator application: float32, float64, or double-float
// (float pairs; maps and outputs in float64, the input map pre-split into pairs).
enum { OPP_F32 = 0, OPP_F64 = 1, OPP_DF64 = 2 };
// IN_RESID: the residual timestream d - A x of the map `in` and the float
// timestream Plan::resid_d (resid_stride floats per right-hand side).
enum { IN_MAP = 0, IN_TOD = 1, IN_TOD_REAL = 2, IN_RESID = 3 };
enum { OUT_MAP = 0, OUT_TOD = 1 };

// Runs the three-kernel noise-weighting pipeline over the plan's tiles with
// input taken from a map (gather, y = A x) or a timestream, and output
// scattered into a map (A^T w, accumulated: caller zeroes it) or written to a
// timestream.  in/out element types follow `prec` (OPP_DF64: input map of
// df64 pairs or float timestream, output float64 map).  `skip` (device int, may be
// NULL) makes every kernel return at once when non-zero.  n_rhs == 0 only sets
// kernel attributes (call it before a stream capture).
madmap_status op_launch(Plan* p, int prec, int in_mode, int out_mode, const void* in, void* out,
                        long long in_stride, long long out_stride, int n_rhs, const int* skip,
                        cudaStream_t s);

size_t f1_smem_bytes(const Plan* p, int prec);

// Event timing of the map-to-map operator: ms[0..2] mean duration of one
// launch of each kernel (chunks run one after another on `s`), ms[3] mean
// duration of one application as the solver launches it.
madmap_status op_time(Plan* p, int prec, const void* in, void* out, int reps, double ms[4], cudaStream_t s);

// Resident CTAs per SM of the operator kernels and CTAs per tile.
void op_occupancy(const Plan* p, int prec, int& ctas_per_sm, int& ctas_per_tile);

// Number of operator launches per application and tiles per launch.
void chunking(const Plan* p, int& n_chunks, int& per_chunk, int n_tiles = -1);

// The operator over a tile set (lanes carry their rhs; per-rhs strides in
// elements; skip[rhs * skip_stride], if skip is not NULL, marks right-hand
// sides whose tiles need no work).
madmap_status op_launch_set(Plan* p, int prec, int in_mode, int out_mode, const void* in, void* out,
                            long long in_stride, long long out_stride, const int* skip, int skip_stride,
                            const TileSet* ts, cudaStream_t s);

// Kernel launch accounting (library-wide).
void count_launches(long long n);

// The operator of one precision (float32, float64 or double-float), each
// compiled in its own translation unit; operator.cu picks the table by `prec`.
struct OpImpl {
  madmap_status (*launch)(Plan* p, int in_mode, int out_mode, const void* in, void* out, long long in_stride,
                          long long out_stride, int n_rhs, const int* skip, cudaStream_t s);
  madmap_status (*launch_set)(Plan* p, int in_mode, int out_mode, const void* in, void* out, long long in_stride,
                              long long out_stride, const int* skip, int skip_stride, const TileSet* ts,
                              cudaStream_t s);
  madmap_status (*time)(Plan* p, const void* in, void* out, int reps, double ms[4], cudaStream_t s);
  void (*occupancy)(const Plan* p, int& ctas_per_sm, int& ctas_per_tile);  // NULL for double-float
  size_t (*f13_smem)(const Plan* p);
  // the (cos 2psi, sin 2psi) weights of n angles as this precision's kernels form them
  madmap_status (*weights)(long long n, const float* psi, void* c, void* s, cudaStream_t st);
};
const OpImpl& op_impl_f32();
const OpImpl& op_impl_f64();
const OpImpl& op_impl_df64();

// Overlap-save windows of the intervals [off[i], off[i+1]) for FFT length M,
// paired two per complex FFT within each filter.
void build_tiles(const std::vector<long long>& off, const std::vector<int>& filt, int n_filters, int n_lags, int M,
                 std::vector<Tile>& tiles);

// Tile set for n_rhs right-hand sides (cached in the plan).
madmap_status get_tile_set(Plan* p, int n_rhs, TileSet** out);

// Deterministic plans: a timestream buffer for n_rhs right-hand sides.
madmap_status ensure_wtod(Plan* p, int n_rhs);

// host FFT (radix 2, float64), used at plan time only
void host_fft(std::vector<double>& re, std::vector<double>& im, bool inverse);

// ---------------------------------------------------------------- device helpers
__host__ __device__ inline int ilog2(unsigned v) {
  int r = 0;
  while ((1u << r) < v) ++r;
  return r;
}

template <typename R> struct CxT;
template <> struct CxT<float> { typedef float2 type; };
template <> struct CxT<double> { typedef double2 type; };
template <> struct CxT<df64> { typedef cdf64 type; };
// Element type of the maps and timestreams an operator instance writes.
template <typename R> struct OutT { typedef R type; };
template <> struct OutT<df64> { typedef double type; };

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename C>
__device__ __forceinline__ C cmulc(C a, C b) {  // a * conj(b)
  C r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.y * b.x - a.x * b.y;
  return r;
}
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) {
  C r;
  r.x = a.x + b.x;
  r.y = a.y + b.y;
  return r;
}
template <typename C>
__device__ __forceinline__ C csub(C a, C b) {
  C r;
  r.x = a.x - b.x;
  r.y = a.y - b.y;
  return r;
}

// Shared-memory layout of the FFT buffers.  Rows sit `rs` elements apart and
// element i of a row is stored at swz<SW>(i): bits 0-3 of i XORed with bits
// 3-6 (SW = 0) or with bits 3-6 XOR bits 4-7 (SW = 1).  Both maps permute
// each aligned block of 16 elements, so a row of N elements fills exactly N
// slots.  The variant and the row padding for each transform length come from
// a bank model of every load, butterfly and store phase of the kernel: with
// them each warp access needs the minimum number of wavefronts (128 bytes
// each) for 8- and 16-byte elements.
template <int SW>
__device__ __forceinline__ int swz(int i) {
  return SW == 0 ? (i ^ ((i >> 3) & 15)) : (i ^ (((i >> 3) ^ (i >> 4)) & 15));
}
// Variant and row stride for transforms of length 2^lg over complex elements
// of esz bytes; `cols` selects the column kernels (k_f1, k_f3), whose load and
// store phases walk down several rows at once, over the row kernel (k_f2).
__host__ __device__ constexpr int lay_sw(int esz, int lg, bool cols) {
  return cols ? ((esz == 16 || lg == 9) ? 0 : 1) : ((esz == 8 && lg == 9) ? 0 : 1);
}
__host__ __device__ constexpr int lay_rs(int esz, int lg, bool cols) {
  return (1 << lg) + (cols ? (lg <= 8 ? 1 : (lg == 9 ? 2 : 4)) : ((esz == 8 && lg <= 6) ? 8 : 0));
}

// Threads per CTA of the operator kernels (every launch uses this many).
constexpr int OP_THREADS = 256;

// Multiplication by the constant w8^k = exp(-2 pi i k / 8), k = 0..3, or its
// conjugate, written out so no general complex product is spent on it.
template <int K, bool CONJ, typename C>
__device__ __forceinline__ C mul_w8(C v) {
  typedef decltype(v.x) R;
  constexpr R h = R(0.70710678118654752440);
  C r;
  if (K == 0) return v;
  if (K == 2) {  // -i (conj: +i)
    if (!CONJ) { r.x = v.y; r.y = -v.x; } else { r.x = -v.y; r.y = v.x; }
    return r;
  }
  if (K == 1) {  // (1 - i)/sqrt2 (conj: (1 + i)/sqrt2)
    if (!CONJ) { r.x = (v.x + v.y) * h; r.y = (v.y - v.x) * h; } else { r.x = (v.x - v.y) * h; r.y = (v.x + v.y) * h; }
    return r;
  }
  // K == 3: (-1 - i)/sqrt2 (conj: (-1 + i)/sqrt2)
  if (!CONJ) { r.x = (v.y - v.x) * h; r.y = -(v.x + v.y) * h; } else { r.x = -(v.x + v.y) * h; r.y = (v.x - v.y) * h; }
  return r;
}

template <int R>
__device__ __forceinline__ constexpr int brev_small(int m) {
  return R == 1 ? m : (R == 2 ? (((m & 1) << 1) | (m >> 1)) : (((m & 1) << 2) | (m & 2) | (m >> 2)));
}

// 2^R-point DFT of v in registers with the output in bit-reversed order
// (R radix-2 decimation-in-frequency stages with constant twiddles), or its
// exact inverse (input in bit-reversed order, unnormalised).
template <typename C, int R, bool INV>
__device__ __forceinline__ void small_dft(C (&v)[1 << R]) {
  if (!INV) {
#pragma unroll
    for (int st = 0; st < R; ++st) {
      const int span = 1 << (R - 1 - st);
#pragma unroll
      for (int m = 0; m < (1 << R); ++m) {
        if ((m & span) == 0) {
          const C x = v[m], y = v[m + span];
          const C d = csub(x, y);
          v[m] = cadd(x, y);
          const int k8 = ((m & (span - 1)) << st) << (3 - R);
          v[m + span] = k8 == 0 ? d : (k8 == 1 ? mul_w8<1, false>(d) : (k8 == 2 ? mul_w8<2, false>(d) : mul_w8<3, false>(d)));
        }
      }
    }
  } else {
#pragma unroll
    for (int st = R - 1; st >= 0; --st) {
      const int span = 1 << (R - 1 - st);
#pragma unroll
      for (int m = 0; m < (1 << R); ++m) {
        if ((m & span) == 0) {
          const int k8 = ((m & (span - 1)) << st) << (3 - R);
          const C b = v[m + span];
          const C y = k8 == 0 ? b : (k8 == 1 ? mul_w8<1, true>(b) : (k8 == 2 ? mul_w8<2, true>(b) : mul_w8<3, true>(b)));
          const C x = v[m];
          v[m] = cadd(x, y);
          v[m + span] = csub(x, y);
        }
      }
    }
  }
}

// Group geometry of a pass: R radix-2 stages starting at stage s of an
// N = 2^logN transform; group g of a row owns the 2^R elements
// base + m * hR (m = 0 .. 2^R - 1) and its output twiddles are
// exp(-2 pi i (j << s) k / N) for k = brev_R(m).  They are read from the
// pass's own table twp[(k - 1) * hR + j] (see build_pass_twiddles), so the
// threads of a warp read consecutive entries.
struct PassGeom {
  int logh, hR, gpr_log;
  __device__ __forceinline__ PassGeom(int logN, int s, int R) {
    logh = logN - s - R;
    hR = 1 << logh;
    gpr_log = logN - R;
  }
  __device__ __forceinline__ void group(int g, int R, int& row, int& base, int& j) const {
    row = g >> gpr_log;
    const int gr = g & ((1 << gpr_log) - 1);
    const int blk = gr >> logh;
    j = gr & (hR - 1);
    base = (blk << (logh + R)) + j;
  }
};

// One radix-2^R pass (R = 1..3) over `rows` rows held in shared memory:
// forward = small DFT then output twiddles (decimation in frequency, output
// bit-reversed after all passes); inverse = conjugate twiddles then inverse
// small DFT, passes in reverse order, returning N times the input.
// The output twiddles w^k (k = 1 .. 2^R - 1) of a group, w = tw[j] the k = 1
// entry of its pass table.  Float32 forms them by products of w (w^2 = w w,
// w^3 = w^2 w, w^4 = w^2 w^2, w^5 = w^4 w, w^6 = w^3 w^3, w^7 = w^4 w^3: at most
// three roundings past the table entry), so a group reads one table entry
// instead of 2^R - 1 and the shared-memory pipe, which bounds the operator
// kernels, carries less; the float64-size types read every power from the
// table (their products cost more than the loads).
#ifndef MM_TW_POWERS
#define MM_TW_POWERS 1
#endif
template <typename C, int R>
__device__ __forceinline__ void pass_twiddles(const C* tw, int logh, int j, C (&w)[1 << R]) {
  if constexpr (sizeof(C) == 8 && MM_TW_POWERS) {
    w[1] = tw[j];
    if (R >= 2) {
      w[2] = cmul(w[1], w[1]);
      w[3] = cmul(w[2], w[1]);
    }
    if (R >= 3) {
      w[4] = cmul(w[2], w[2]);
      w[5] = cmul(w[4], w[1]);
      w[6] = cmul(w[3], w[3]);
      w[7] = cmul(w[4], w[3]);
    }
  } else {
#pragma unroll
    for (int k = 1; k < (1 << R); ++k) w[k] = tw[((k - 1) << logh) + j];
  }
}

template <typename C, int R, bool INV, int SW>
__device__ __forceinline__ void fft_pass(C* buf, int rows, int rs, int logN, int s, const C* tw) {
  const PassGeom G(logN, s, R);
  const int total = rows << G.gpr_log;
#pragma unroll 4
  for (int g = threadIdx.x; g < total; g += OP_THREADS) {
    int row, base, j;
    G.group(g, R, row, base, j);
    C* rp = buf + row * rs;
    C v[1 << R];
#pragma unroll
    for (int m = 0; m < (1 << R); ++m) v[m] = rp[swz<SW>(base + m * G.hR)];
    C w[1 << R];
    pass_twiddles<C, R>(tw, G.logh, j, w);
    if (!INV) {
      small_dft<C, R, false>(v);
#pragma unroll
      for (int m = 1; m < (1 << R); ++m) v[m] = cmul(v[m], w[brev_small<R>(m)]);
    } else {
#pragma unroll
      for (int m = 1; m < (1 << R); ++m) v[m] = cmulc(v[m], w[brev_small<R>(m)]);
      small_dft<C, R, true>(v);
    }
#pragma unroll
    for (int m = 0; m < (1 << R); ++m) rp[swz<SW>(base + m * G.hR)] = v[m];
  }
}

__host__ __device__ constexpr int last_pass_start(int logN) { return ((logN - 1) / 3) * 3; }

// Offset of pass s's twiddle table: passes before it hold (2^R - 1) N/2^(s'+R)
// entries each (N - 1 entries in all).
__device__ __forceinline__ int pass_offset(int logN, int s) {
  int off = 0;
  for (int q = 0; q < s; q += 3) {
    const int R = (logN - q) >= 3 ? 3 : (logN - q);
    off += ((1 << R) - 1) << (logN - q - R);
  }
  return off;
}

// Per-pass output-twiddle tables of an N = 2^logN transform, from the plan's
// table twM (exp(-2 pi i j / M), read with stride M/N): entry (k - 1) * hR + j
// of pass s is exp(-2 pi i (j << s) k / N).
template <typename C>
__device__ __forceinline__ void build_pass_twiddles(C* twp, int logN, const C* twM, long long stride) {
  int off = 0;
  for (int s = 0; s < logN; s += 3) {
    const int R = (logN - s) >= 3 ? 3 : (logN - s);
    const int logh = logN - s - R;
    const int cnt = ((1 << R) - 1) << logh;
    for (int i = threadIdx.x; i < cnt; i += OP_THREADS) {
      const int k = (i >> logh) + 1, j = i & ((1 << logh) - 1);
      twp[off + i] = twM[(long long)((j << s) * k) * stride];
    }
    off += cnt;
  }
}

template <typename C, bool INV, int SW>
__device__ __forceinline__ void fft_pass_any(C* buf, int rows, int rs, int logN, int s, const C* tw) {
  const int R = (logN - s) >= 3 ? 3 : (logN - s);
  const C* twp = tw + pass_offset(logN, s);
  if (R == 3) fft_pass<C, 3, INV, SW>(buf, rows, rs, logN, s, twp);
  else if (R == 2) fft_pass<C, 2, INV, SW>(buf, rows, rs, logN, s, twp);
  else fft_pass<C, 1, INV, SW>(buf, rows, rs, logN, s, twp);
}

// Full FFT of `rows` rows of length N = 2^logN held in shared memory
// (tw: N entries).  s_lo = 3 leaves out the first pass (s = 0) of a forward
// transform, or the last pass of an inverse one, which the caller does in
// registers (reg_pass8).
// s_hi < 0 (the default) runs every pass up to the last; s_hi = the last
// pass's start leaves it out (forward: the last pass; inverse: the first),
// for the caller to do it in registers (reg_pass_last).
template <typename C, bool INV, int SW>
__device__ __forceinline__ void fft_rows(C* buf, int rows, int rs, int logN, const C* tw, int s_lo = 0,
                                         int s_hi = -1) {
  const int top = s_hi < 0 ? last_pass_start(logN) + 3 : s_hi;
  if (!INV) {
#pragma unroll
    for (int s = s_lo; s < top; s += 3) {
      fft_pass_any<C, false, SW>(buf, rows, rs, logN, s, tw);
      __syncthreads();
    }
  } else {
#pragma unroll
    for (int s = top - 3; s >= s_lo; s -= 3) {
      fft_pass_any<C, true, SW>(buf, rows, rs, logN, s, tw);
      __syncthreads();
    }
  }
}

// The last pass of a forward transform (radix 2^R on 2^R consecutive
// elements; its twiddles are all 1) on one group held in registers, or, INV,
// the first pass of the inverse transform.
template <typename C, int R, bool INV>
__device__ __forceinline__ void reg_pass_last(C (&v)[1 << R]) {
  small_dft<C, R, INV>(v);
}

// The first radix-8 pass (s = 0) of a forward transform of length N on one
// group held in registers: the elements base + m N/8 (m = 0..7) in v, the
// group's twiddles from the pass table entry tw[base]; or, INV, the last pass
// of the inverse transform.  The same arithmetic as fft_pass<C, 3, INV> on the
// group, with no trip through shared memory.
template <typename C, bool INV>
__device__ __forceinline__ void reg_pass8(C (&v)[8], const C* tw, int logN, int base) {
  C w[8];
  pass_twiddles<C, 3>(tw, logN - 3, base, w);
  if (!INV) {
    small_dft<C, 3, false>(v);
#pragma unroll
    for (int m = 1; m < 8; ++m) v[m] = cmul(v[m], w[brev_small<3>(m)]);
  } else {
#pragma unroll
    for (int m = 1; m < 8; ++m) v[m] = cmulc(v[m], w[brev_small<3>(m)]);
    small_dft<C, 3, true>(v);
  }
}

// Forward FFT, pointwise product with a real spectrum and inverse FFT of
// `rows` rows: the last forward pass, the product and the first inverse pass
// act on the same element groups, so they run back to back in registers.
// Hrow(row) points at the row's spectrum (bit-reversed order, as the forward
// transform leaves it).
template <typename C, int R, int SW, typename HF>
__device__ __forceinline__ void fused_middle(C* buf, int rows, int rs, int logN, int s, HF Hrow) {
  typedef decltype(C().x) Real;
  const PassGeom G(logN, s, R);
  const int total = rows << G.gpr_log;
#pragma unroll 4
  for (int g = threadIdx.x; g < total; g += OP_THREADS) {
    int row, base, j;
    G.group(g, R, row, base, j);
    C* rp = buf + row * rs;
    const Real* H = Hrow(row);
    C v[1 << R];
    Real hv[1 << R];
#pragma unroll
    for (int m = 0; m < (1 << R); ++m) {
      v[m] = rp[swz<SW>(base + m * G.hR)];
      hv[m] = H[base + m * G.hR];
    }
    // The forward pass ends with output twiddles w and the inverse pass starts
    // with their conjugates; |w| = 1, so between the two small DFTs only the
    // filter product remains.
    small_dft<C, R, false>(v);
#pragma unroll
    for (int m = 0; m < (1 << R); ++m) {
      v[m].x *= hv[m];
      v[m].y *= hv[m];
    }
    small_dft<C, R, true>(v);
#pragma unroll
    for (int m = 0; m < (1 << R); ++m) rp[swz<SW>(base + m * G.hR)] = v[m];
  }
}

template <typename C, int SW, typename HF>
__device__ __forceinline__ void fft_rows_filter(C* buf, int rows, int rs, int logN, const C* tw, HF Hrow,
                                                int s_lo = 0) {
  const int sl = last_pass_start(logN);
#pragma unroll
  for (int s = s_lo; s < sl; s += 3) {
    fft_pass_any<C, false, SW>(buf, rows, rs, logN, s, tw);
    __syncthreads();
  }
  const int R = logN - sl;
  if (R == 3) fused_middle<C, 3, SW>(buf, rows, rs, logN, sl, Hrow);
  else if (R == 2) fused_middle<C, 2, SW>(buf, rows, rs, logN, sl, Hrow);
  else fused_middle<C, 1, SW>(buf, rows, rs, logN, sl, Hrow);
  __syncthreads();
#pragma unroll
  for (int s = sl - 3; s >= s_lo; s -= 3) {
    fft_pass_any<C, true, SW>(buf, rows, rs, logN, s, tw);
    __syncthreads();
  }
}

__device__ __forceinline__ int brev_n(int v, int bits) {
  return bits == 0 ? 0 : (int)(__brev((unsigned)v) >> (32 - bits));
}

}  // namespace mm
