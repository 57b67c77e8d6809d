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
  void* scratch = nullptr;         // tiles_per_chunk * M complex (float64 size)
  int* dev_flag = nullptr;         // small device flag words
  size_t device_bytes = 0;
  std::vector<void*> allocs;
  SolveBuffers* sb64 = nullptr;
  SolveBuffers* sb32 = nullptr;
  // solves run on a plan-owned non-blocking stream (graph capture is not
  // allowed on the legacy default stream), ordered after the caller's stream
  cudaStream_t solve_stream = nullptr;
  cudaEvent_t solve_event = nullptr;
  ~Plan();
};

madmap_status dalloc(Plan* p, void** ptr, size_t bytes);
template <typename T>
inline madmap_status dalloc_t(Plan* p, T** ptr, size_t count) {
  return dalloc(p, reinterpret_cast<void**>(ptr), count * sizeof(T));
}

// ---------------------------------------------------------------- operator launch
enum { IN_MAP = 0, IN_TOD = 1, IN_TOD_REAL = 2 };
enum { OUT_MAP = 0, OUT_TOD = 1 };

// Runs the three-kernel noise-weighting pipeline over the plan's tiles with
// input taken from a map (gather, y = A x) or a timestream, and output
// scattered into a map (A^T w, accumulated: caller zeroes it) or written to a
// timestream.  in/out element types follow `fp64`.  `skip` (device int, may be
// NULL) makes every kernel return at once when non-zero.  n_rhs == 0 only sets
// kernel attributes (call it before a stream capture).
madmap_status op_launch(Plan* p, bool fp64, int in_mode, int out_mode, const void* in, void* out,
                        long long in_stride, long long out_stride, int n_rhs, const int* skip,
                        cudaStream_t s);

size_t f1_smem_bytes(const Plan* p, bool fp64);

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

// Shared-memory row layout: one padding element every 32 keeps strided
// butterfly accesses off a single bank; rows are an odd number of elements
// apart so column-wise accesses spread over the banks.
__device__ __forceinline__ int sidx(int i) { return i + (i >> 5); }
__host__ __device__ inline int row_stride(int n) { return n + (n >> 5) + 1; }

// One pass of in-place radix-2 decimation-in-frequency (forward) or
// decimation-in-time (inverse, conjugate twiddles) stages, R = 1..3 stages fused
// in registers.  `s` is the index of the first stage; stage s has span
// N >> (s+1).  Each thread owns groups of 2^R elements spaced hR = N >> (s+R)
// apart.  tw[k] = exp(-2 pi i k / N), k < N/2.  Forward passes run s = 0, 3,
// 6, ...; the output is in bit-reversed order.  The inverse runs the same
// passes in reverse order and returns N times the input.
template <typename C, int R, bool INV>
__device__ __forceinline__ void fft_pass(C* buf, int rows, int rs, int logN, int s, const C* tw) {
  const int logh = logN - s - R;
  const int hR = 1 << logh;
  const int gpr_log = logN - R;  // groups per row = N >> R
  const int total = rows << gpr_log;
  for (int g = threadIdx.x; g < total; g += blockDim.x) {
    const int row = g >> gpr_log;
    const int gr = g & ((1 << gpr_log) - 1);
    const int blk = gr >> logh;
    const int j = gr & (hR - 1);
    const int base = (blk << (logh + R)) + j;
    C* rp = buf + row * rs;
    C v[1 << R];
#pragma unroll
    for (int m = 0; m < (1 << R); ++m) v[m] = rp[sidx(base + m * hR)];
    if (!INV) {
#pragma unroll
      for (int st = 0; st < R; ++st) {
        const int span = 1 << (R - 1 - st);
#pragma unroll
        for (int m = 0; m < (1 << R); ++m) {
          if ((m & span) == 0) {
            const int pos = j + (m & (span - 1)) * hR;
            const C w = tw[pos << (s + st)];
            const C x = v[m], y = v[m + span];
            v[m] = cadd(x, y);
            v[m + span] = cmul(csub(x, y), w);
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
            const int pos = j + (m & (span - 1)) * hR;
            const C w = tw[pos << (s + st)];
            const C x = v[m];
            const C y = cmulc(v[m + span], w);
            v[m] = cadd(x, y);
            v[m + span] = csub(x, y);
          }
        }
      }
    }
#pragma unroll
    for (int m = 0; m < (1 << R); ++m) rp[sidx(base + m * hR)] = v[m];
  }
}

// Full FFT of `rows` rows of length N = 2^logN held in shared memory.
template <typename C, bool INV>
__device__ void fft_rows(C* buf, int rows, int rs, int logN, const C* tw) {
  if (!INV) {
    for (int s = 0; s < logN; s += 3) {
      const int R = (logN - s) >= 3 ? 3 : (logN - s);
      if (R == 3) fft_pass<C, 3, false>(buf, rows, rs, logN, s, tw);
      else if (R == 2) fft_pass<C, 2, false>(buf, rows, rs, logN, s, tw);
      else fft_pass<C, 1, false>(buf, rows, rs, logN, s, tw);
      __syncthreads();
    }
  } else {
    int last = ((logN - 1) / 3) * 3;
    for (int s = last; s >= 0; s -= 3) {
      const int R = (logN - s) >= 3 ? 3 : (logN - s);
      if (R == 3) fft_pass<C, 3, true>(buf, rows, rs, logN, s, tw);
      else if (R == 2) fft_pass<C, 2, true>(buf, rows, rs, logN, s, tw);
      else fft_pass<C, 1, true>(buf, rows, rs, logN, s, tw);
      __syncthreads();
    }
  }
}

__device__ __forceinline__ int brev_n(int v, int bits) {
  return bits == 0 ? 0 : (int)(__brev((unsigned)v) >> (32 - bits));
}

}  // namespace mm
