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
//
// This file holds the precision-independent entry points and the
// allocation-free weighting; the kernels are in operator_kernels.cuh.
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace mm {

// Tiles are processed in n_chunks launches of (nearly) equal size, at most
// tiles_per_chunk each, so no launch is left with a small tail of work.
void chunking(const Plan* p, int& n_chunks, int& per_chunk, int n_tiles) {
  if (n_tiles < 0 && p->diag) {  // one diagonal pass per application
    n_chunks = p->n_tiles ? 1 : 0;
    per_chunk = p->n_tiles;
    return;
  }
  if (n_tiles < 0) n_tiles = p->n_tiles;
  n_chunks = n_tiles ? (n_tiles + p->tiles_per_chunk - 1) / p->tiles_per_chunk : 0;
  per_chunk = n_chunks ? (n_tiles + n_chunks - 1) / n_chunks : 0;
}


static const OpImpl& impl_for(int prec) {
  return prec == OPP_DF64 ? op_impl_df64() : prec == OPP_F64 ? op_impl_f64() : op_impl_f32();
}

// Operator over a tile set whose lanes name their right-hand side (maps and
// timestreams strided by in_stride / out_stride elements per rhs).
madmap_status op_launch_set(Plan* p, int prec, int in_mode, int out_mode, const void* in, void* out,
                            long long in_stride, long long out_stride, const int* skip, int skip_stride,
                            const TileSet* ts, cudaStream_t s) {
  if (ts->n_tiles == 0) return MADMAP_OK;
  return impl_for(prec).launch_set(p, in_mode, out_mode, in, out, in_stride, out_stride, skip, skip_stride, ts, s);
}

static long long g_launches = 0;
void count_launches(long long n) { g_launches += n; }

madmap_status op_time(Plan* p, int prec, const void* in, void* out, int reps, double ms[4], cudaStream_t s) {
  if (p->n_tiles == 0) {
    ms[0] = ms[1] = ms[2] = ms[3] = 0.0;
    return MADMAP_OK;
  }
  return impl_for(prec).time(p, in, out, reps, ms, s);
}

// The float64 kernels' occupancy stands for the double-float ones too.
void op_occupancy(const Plan* p, int prec, int& ctas_per_sm, int& ctas_per_tile) {
  (prec == OPP_F32 ? op_impl_f32() : op_impl_f64()).occupancy(p, ctas_per_sm, ctas_per_tile);
}

size_t f1_smem_bytes(const Plan* p, int prec) { return impl_for(prec).f13_smem(p); }

// in_mode: IN_MAP (gather from a map), IN_TOD (float timestream, e.g. the
// data d) or IN_TOD_REAL (timestream of the working precision).  n_rhs == 0
// only prepares the kernels (shared-memory opt-in) and launches nothing.
madmap_status op_launch(Plan* p, int prec, int in_mode, int out_mode, const void* in, void* out,
                        long long in_stride, long long out_stride, int n_rhs, const int* skip,
                        cudaStream_t s) {
  if (p->n_tiles == 0) return MADMAP_OK;
  return impl_for(prec).launch(p, in_mode, out_mode, in, out, in_stride, out_stride, n_rhs, skip, s);
}

}  // namespace mm

extern "C" int64_t madmap_kernel_launch_count(void) { return (int64_t)mm::g_launches; }

extern "C" madmap_status madmap_polarisation_weights(int32_t precision, int64_t n, const float* psi, void* cos2psi,
                                                     void* sin2psi, void* stream) {
  using namespace mm;
  MM_CHECK(precision == MADMAP_FP32 || precision == MADMAP_FP64, MADMAP_ERR_INVALID_ARG,
           "polarisation_weights: precision must be FP32 or FP64");
  MM_CHECK(n >= 0, MADMAP_ERR_INVALID_ARG, "polarisation_weights: n < 0");
  if (n == 0) return MADMAP_OK;
  MM_CHECK(psi && cos2psi && sin2psi, MADMAP_ERR_INVALID_ARG, "polarisation_weights: NULL pointer");
  const OpImpl& impl = precision == MADMAP_FP32 ? op_impl_f32() : op_impl_f64();
  return impl.weights(n, psi, cos2psi, sin2psi, static_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------------- allocation-free noise weighting
// Some callers cannot allocate device memory at the point where they need the
// noise weighting: code running under an allocator that forbids new device
// allocations after start-up, real-time loops that must not stall on
// cudaMalloc, or host code that owns no CUDA memory management of its own.
// madmap_apply_ninv_noalloc serves them: it runs the same three weighting
// kernels as madmap_apply_ninv, but every derived buffer (twiddles, filter
// spectra, window descriptors and the FFT intermediate) lives in the fixed
// array below, which every GPU that loads the library holds until the
// process exits.  The caller passes inputs and outputs only.
//
// The array is shared by all calls: each call rewrites the parts it reads
// (nothing needs to start at zero), and calls that overlap on the GPU (on
// different streams, or from different host threads) race on it.  Each call
// looks up the array's device address for the device that is current, so
// the address stays right after a device reset.  The derived tables are
// uploaded from host memory that lives only for the duration of the call, so
// the call refuses to be recorded into a CUDA graph (a replay would read
// freed host memory), and the upload may hold the host until the stream has
// reached it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MADMAP_NOALLOC_SCRATCH_BYTES];

namespace mm {
namespace {

// The array's device address on the current device (a host-side lookup; the
// name g_noalloc_scratch is only a host stand-in and must not be handed to a
// kernel).
madmap_status noalloc_scratch(void** out) {
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
  *out = ptr;
  return MADMAP_OK;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace
}  // namespace mm

extern "C" madmap_status madmap_apply_ninv_noalloc(int32_t precision, int64_t n_samples, int32_t n_intervals,
                                                   const int64_t* interval_offsets, const int32_t* interval_filter,
                                                   int32_t n_filters, int32_t n_lags, const double* filter_lags,
                                                   const void* y, void* w, void* stream) {
  using namespace mm;
  MM_CHECK(precision == MADMAP_FP64 || precision == MADMAP_FP32, MADMAP_ERR_INVALID_ARG,
           "apply_ninv_noalloc: precision must be FP64 or FP32");
  MM_CHECK(n_samples >= 0 && n_intervals >= 0 && interval_offsets, MADMAP_ERR_INVALID_ARG,
           "apply_ninv_noalloc: bad sizes or offsets");
  MM_CHECK(n_intervals == 0 || interval_filter, MADMAP_ERR_INVALID_ARG, "apply_ninv_noalloc: interval_filter NULL");
  MM_CHECK(n_filters >= 1 && n_lags >= 1 && filter_lags, MADMAP_ERR_INVALID_ARG,
           "apply_ninv_noalloc: need n_filters >= 1, n_lags >= 1 and filter_lags");
  MM_CHECK(interval_offsets[0] == 0 && interval_offsets[n_intervals] == n_samples, MADMAP_ERR_INVALID_ARG,
           "apply_ninv_noalloc: interval_offsets must start at 0 and end at n_samples");
  for (int i = 0; i < n_intervals; ++i) {
    MM_CHECK(interval_offsets[i + 1] >= interval_offsets[i], MADMAP_ERR_INVALID_ARG,
             "apply_ninv_noalloc: interval_offsets must be non-decreasing");
    MM_CHECK(interval_filter[i] >= 0 && interval_filter[i] < n_filters, MADMAP_ERR_INVALID_ARG,
             "apply_ninv_noalloc: interval_filter out of range");
  }
  for (long long k = 0; k < (long long)n_filters * n_lags; ++k)
    MM_CHECK(isfinite(filter_lags[k]), MADMAP_ERR_INVALID_ARG, "apply_ninv_noalloc: filter_lags must be finite");
  MM_CHECK(n_lags <= MADMAP_NOALLOC_MAX_LAGS, MADMAP_ERR_INVALID_ARG,
           "apply_ninv_noalloc: n_lags above the limit of the fixed scratch (MADMAP_NOALLOC_MAX_LAGS)");
  if (n_samples == 0) return MADMAP_OK;
  MM_CHECK(y && w, MADMAP_ERR_INVALID_ARG, "apply_ninv_noalloc: NULL timestream");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    MM_CUDA(cudaStreamIsCapturing(s, &cs));
    MM_CHECK(cs == cudaStreamCaptureStatusNone, MADMAP_ERR_INVALID_ARG,
             "apply_ninv_noalloc: cannot be recorded by a stream capture (its tables are uploaded from host "
             "memory that does not outlive the call)");
  }
  const bool fp64 = precision == MADMAP_FP64;
  // FFT length: four bandwidths per window, so at least half of every window
  // is exact output
  int M = 256;
  while (M < 4 * n_lags) M <<= 1;
  Plan q;  // describes the launch only; owns no memory
  q.n_stokes = 1;
  q.ns_pad = 1;
  q.n_t = n_samples;
  q.n_filters = n_filters;
  q.n_lags = n_lags;
  q.M = M;
  {
    const int lg = ilog2((unsigned)M);
    q.logN2 = (lg + 1) / 2;
    q.logN1 = lg - q.logN2;
    q.N1 = 1 << q.logN1;
    q.N2 = 1 << q.logN2;
  }
  std::vector<long long> off(interval_offsets, interval_offsets + n_intervals + 1);
  std::vector<int> filt(interval_filter, interval_filter + n_intervals);
  std::vector<Tile> tiles;
  build_tiles(off, filt, n_filters, n_lags, M, tiles);
  q.n_tiles = (int)tiles.size();
  const size_t ce = fp64 ? sizeof(double2) : sizeof(float2), re = fp64 ? sizeof(double) : sizeof(float);
  const size_t off_tw = 0;
  const size_t off_H = align256(off_tw + (size_t)M * ce);
  const size_t off_T = align256(off_H + (size_t)n_filters * M * re);
  const size_t off_S = align256(off_T + tiles.size() * sizeof(Tile));
  const size_t per_tile = (size_t)M * ce;
  MM_CHECK(off_S + per_tile <= (size_t)MADMAP_NOALLOC_SCRATCH_BYTES, MADMAP_ERR_INVALID_ARG,
           "apply_ninv_noalloc: filters and windows exceed the fixed scratch (MADMAP_NOALLOC_SCRATCH_BYTES)");
  const long long cap = (long long)(((size_t)MADMAP_NOALLOC_SCRATCH_BYTES - off_S) / per_tile);
  q.tiles_per_chunk = (int)std::max(1LL, std::min<long long>(std::min<long long>(cap, 65535), std::max(1, q.n_tiles)));
  // host-side tables: twiddles exp(-2 pi i j / M) and the permuted circulant spectra / M
  std::vector<double> h64((size_t)n_filters * M);
  std::vector<double> re_(M), im_(M);
  for (int f = 0; f < n_filters; ++f) {
    std::fill(re_.begin(), re_.end(), 0.0);
    std::fill(im_.begin(), im_.end(), 0.0);
    const double* lg = filter_lags + (size_t)f * n_lags;
    re_[0] = lg[0];
    for (int t = 1; t < n_lags; ++t) {
      re_[t] += lg[t];
      re_[M - t] += lg[t];
    }
    host_fft(re_, im_, false);
    double mn = 1e300;
    for (int k = 0; k < M; ++k) mn = std::min(mn, re_[k]);
    MM_CHECK(mn > 0.0, MADMAP_ERR_NOT_PD, "apply_ninv_noalloc: a filter is not positive definite");
    for (int p2 = 0; p2 < q.N2; ++p2) {
      int k2 = 0;
      for (int b = 0; b < q.logN2; ++b) k2 |= ((p2 >> b) & 1) << (q.logN2 - 1 - b);
      for (int p1 = 0; p1 < q.N1; ++p1) {
        int k1 = 0;
        for (int b = 0; b < q.logN1; ++b) k1 |= ((p1 >> b) & 1) << (q.logN1 - 1 - b);
        h64[(size_t)f * M + (size_t)p2 * q.N1 + p1] = re_[k2 + (size_t)q.N2 * k1] / (double)M;
      }
    }
  }
  void* base = nullptr;
  madmap_status st = noalloc_scratch(&base);
  if (st != MADMAP_OK) return st;
  unsigned char* b = static_cast<unsigned char*>(base);
  if (fp64) {
    std::vector<double2> t64(M);
    for (int j = 0; j < M; ++j) {
      const double ang = 2.0 * M_PI * (double)j / (double)M;
      t64[j] = make_double2(cos(ang), -sin(ang));
    }
    MM_CUDA(cudaMemcpyAsync(b + off_tw, t64.data(), (size_t)M * sizeof(double2), cudaMemcpyHostToDevice, s));
    MM_CUDA(cudaMemcpyAsync(b + off_H, h64.data(), h64.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    q.tw64 = reinterpret_cast<double2*>(b + off_tw);
    q.H64 = reinterpret_cast<double*>(b + off_H);
  } else {
    std::vector<float2> t32(M);
    std::vector<float> h32(h64.size());
    for (int j = 0; j < M; ++j) {
      const double ang = 2.0 * M_PI * (double)j / (double)M;
      t32[j] = make_float2((float)cos(ang), (float)-sin(ang));
    }
    for (size_t k = 0; k < h64.size(); ++k) h32[k] = (float)h64[k];
    MM_CUDA(cudaMemcpyAsync(b + off_tw, t32.data(), (size_t)M * sizeof(float2), cudaMemcpyHostToDevice, s));
    MM_CUDA(cudaMemcpyAsync(b + off_H, h32.data(), h32.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    q.tw32 = reinterpret_cast<float2*>(b + off_tw);
    q.H32 = reinterpret_cast<float*>(b + off_H);
  }
  if (!tiles.empty())
    MM_CUDA(cudaMemcpyAsync(b + off_T, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice, s));
  q.tiles = reinterpret_cast<Tile*>(b + off_T);
  q.scratch = b + off_S;
  if (q.n_tiles == 0) return MADMAP_OK;
  st = op_launch(&q, fp64 ? OPP_F64 : OPP_F32, IN_TOD_REAL, OUT_TOD, y, w, 0, 0, 1, nullptr, s);
  // the host tables above were copied from pageable memory: such a copy has
  // read its source before cudaMemcpyAsync returns, so they may go out of
  // scope here
  return st;
}
