// Plan construction: validation, observed-pixel indexing (Section 5.4), pixel
// classification and block preconditioner (Sections 4-5), overlap-save
// windows and filter spectra (Section 5.2), and the host-side helpers of the
// C ABI (errors, noise-filter lags, the paper's FFT-length rule).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace mm {

// ---------------------------------------------------------------- errors
static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

madmap_status cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string("CUDA error ") + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ") in " + what;
  if (e == cudaErrorMemoryAllocation) return MADMAP_ERR_OOM;
  return MADMAP_ERR_CUDA;
}

// ---------------------------------------------------------------- allocation
// MADMAP_FAULT_ALLOC_FAIL_AT=n makes the n-th device allocation of the process
// (counting from 1) report out-of-memory, so callers' error paths can be
// tested on the host without exhausting a shared GPU.
static long long g_alloc_count = 0;

madmap_status dalloc(Plan* p, void** ptr, size_t bytes) {
  *ptr = nullptr;
  ++g_alloc_count;
  const char* inj = getenv("MADMAP_FAULT_ALLOC_FAIL_AT");
  if (inj && atoll(inj) == g_alloc_count) {
    set_error("injected allocation failure (MADMAP_FAULT_ALLOC_FAIL_AT)");
    return MADMAP_ERR_OOM;
  }
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return cuda_fail(e, "cudaMalloc");
  }
  p->allocs.push_back(*ptr);
  p->device_bytes += bytes;
  return MADMAP_OK;
}

// Device buffers that depend on the FFT length (windows, spectra, twiddles,
// scratch): kept apart so the autotuner can rebuild them for another length.
static madmap_status walloc(Plan* p, void** ptr, size_t bytes) {
  madmap_status st = dalloc(p, ptr, bytes);
  if (st != MADMAP_OK) return st;
  p->allocs.pop_back();
  p->win_allocs.push_back(*ptr);
  p->win_bytes += bytes == 0 ? 16 : bytes;
  return MADMAP_OK;
}
template <typename T>
static madmap_status walloc_t(Plan* p, T** ptr, size_t count) {
  return walloc(p, reinterpret_cast<void**>(ptr), count * sizeof(T));
}

static void free_windows(Plan* p) {
  if (p->win_allocs.empty()) return;
  cudaDeviceSynchronize();
  for (void* a : p->win_allocs) cudaFree(a);
  p->win_allocs.clear();
  p->device_bytes -= p->win_bytes;
  p->win_bytes = 0;
  p->tiles = nullptr;
  p->H64 = nullptr;
  p->H32 = nullptr;
  p->Hdf = nullptr;
  p->tw64 = nullptr;
  p->tw32 = nullptr;
  p->twdf = nullptr;
  p->scratch = nullptr;
}

void free_solve_buffers(Plan* p);          // solver.cu
size_t solve_buffer_bytes(const Plan* p);  // solver.cu

Plan::~Plan() {
  free_solve_buffers(this);
  for (TileSet* t : tile_sets) delete t;
  if (solve_event) cudaEventDestroy(solve_event);
  if (solve_stream) cudaStreamDestroy(solve_stream);
  for (int i = 0; i < 2; ++i) {
    if (op_join[i]) cudaEventDestroy(op_join[i]);
    if (op_stream[i]) cudaStreamDestroy(op_stream[i]);
  }
  if (op_fork) cudaEventDestroy(op_fork);
  for (void* a : allocs) cudaFree(a);
  for (void* a : win_allocs) cudaFree(a);
}

// ---------------------------------------------------------------- host FFT
// Iterative radix-2 Cooley-Tukey, float64; length must be a power of two.
void host_fft(std::vector<double>& re, std::vector<double>& im, bool inverse) {
  const size_t n = re.size();
  for (size_t i = 1, j = 0; i < n; ++i) {
    size_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      std::swap(re[i], re[j]);
      std::swap(im[i], im[j]);
    }
  }
  const double sgn = inverse ? 1.0 : -1.0;
  for (size_t len = 2; len <= n; len <<= 1) {
    const size_t half = len >> 1;
    std::vector<double> wr(half), wi(half);
    for (size_t k = 0; k < half; ++k) {
      const double ang = 2.0 * M_PI * (double)k / (double)len;
      wr[k] = cos(ang);
      wi[k] = sgn * sin(ang);
    }
    for (size_t i = 0; i < n; i += len) {
      for (size_t k = 0; k < half; ++k) {
        const size_t a = i + k, b = a + half;
        const double xr = re[b] * wr[k] - im[b] * wi[k];
        const double xi = re[b] * wi[k] + im[b] * wr[k];
        re[b] = re[a] - xr;
        im[b] = im[a] - xi;
        re[a] += xr;
        im[a] += xi;
      }
    }
  }
}

static bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

// ---------------------------------------------------------------- noise filter
// Inverse DFT of an even real sequence q of length L, first n outputs.
static void even_idft(const std::vector<double>& q, int n, double* out) {
  const size_t L = q.size();
  if (is_pow2((long long)L)) {
    std::vector<double> re(q), im(L, 0.0);
    host_fft(re, im, true);
    for (int t = 0; t < n; ++t) out[t] = re[t] / (double)L;
  } else {
    for (int t = 0; t < n; ++t) {
      double acc = 0.0;
      for (size_t j = 0; j < L; ++j) acc += q[j] * cos(2.0 * M_PI * (double)((j * (size_t)t) % L) / (double)L);
      out[t] = acc / (double)L;
    }
  }
}

}  // namespace mm

using namespace mm;

extern "C" madmap_status madmap_noise_filter(int32_t n_lags, double fs, double sigma, double fknee,
                                             double alpha, double* lags_out, double* dlags_out) {
  MM_CHECK(n_lags >= 1 && lags_out, MADMAP_ERR_INVALID_ARG, "noise_filter: n_lags >= 1 and lags_out required");
  MM_CHECK(fs > 0 && sigma > 0 && fknee >= 0 && isfinite(alpha), MADMAP_ERR_INVALID_ARG,
           "noise_filter: need fs > 0, sigma > 0, fknee >= 0, finite alpha");
  const int L = 4 * n_lags;
  std::vector<double> nu(L), q(L);
  for (int j = 0; j < L; ++j) nu[j] = (double)std::min(j, L - j) * fs / (double)L;
  nu[0] = nu[1];
  for (int j = 0; j < L; ++j) q[j] = 1.0 / (sigma * sigma * (1.0 + pow(fknee / nu[j], alpha)));
  std::vector<double> c(n_lags);
  even_idft(q, n_lags, c.data());
  for (int t = 0; t < n_lags; ++t) lags_out[t] = (1.0 - (double)t / n_lags) * c[t];
  if (dlags_out) {
    std::vector<double> dq(L);
    for (int k = 0; k < 3; ++k) {
      for (int j = 0; j < L; ++j) {
        const double r = pow(fknee / nu[j], alpha);
        if (k == 0) dq[j] = -2.0 * q[j] / sigma;
        else if (k == 1) dq[j] = fknee > 0 ? -q[j] * q[j] * sigma * sigma * alpha * r / fknee : 0.0;
        else dq[j] = fknee > 0 ? -q[j] * q[j] * sigma * sigma * r * log(fknee / nu[j]) : 0.0;
      }
      even_idft(dq, n_lags, c.data());
      for (int t = 0; t < n_lags; ++t) dlags_out[k * n_lags + t] = (1.0 - (double)t / n_lags) * c[t];
    }
  }
  return MADMAP_OK;
}

extern "C" madmap_status madmap_noise_filter_vjp(int32_t n_lags, double fs, double sigma, double fknee, double alpha,
                                                 const double* grad_lags, double* grad_params_out) {
  MM_CHECK(n_lags >= 1 && grad_lags && grad_params_out, MADMAP_ERR_INVALID_ARG, "noise_filter_vjp: bad arguments");
  std::vector<double> lags(n_lags), dl(3 * (size_t)n_lags);
  madmap_status st = madmap_noise_filter(n_lags, fs, sigma, fknee, alpha, lags.data(), dl.data());
  if (st != MADMAP_OK) return st;
  for (int k = 0; k < 3; ++k) {
    double acc = 0.0;
    for (int t = 0; t < n_lags; ++t) acc += dl[(size_t)k * n_lags + t] * grad_lags[t];
    grad_params_out[k] = acc;
  }
  return MADMAP_OK;
}

static double hprime(double nf, double nc) {
  return (1.0 + log(nf)) / (nf - 2 * nc) - nf * log(nf) / ((nf - 2 * nc) * (nf - 2 * nc));
}

extern "C" int64_t madmap_paper_fft_length(int64_t n_lags, int64_t longest) {
  int64_t nf = 1;
  while (nf <= longest) nf *= 2;
  while (nf <= 2 * n_lags) nf *= 2;
  if (hprime((double)nf, (double)n_lags) > 0) {
    while (nf / 2 > 2 * n_lags && hprime((double)(nf / 2), (double)n_lags) >= 0) nf /= 2;
  }
  return nf;
}

extern "C" const char* madmap_last_error(void) { return g_err.c_str(); }
extern "C" const char* madmap_version(void) { return "madmap-gb300 0.1"; }

namespace mm {

// ---------------------------------------------------------------- plan kernels
__global__ void k_validate_pix(const int* pix, long long n, int n_pix, int* bad, int bit) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int g = pix[t];
    if (g < -1 || g >= n_pix) atomicOr(bad, bit);
  }
}

__global__ void k_validate_psi(const float* psi, long long n, int* bad) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    if (!isfinite(psi[t])) atomicOr(bad, 2);
  }
}

// Section 5.4: one bit per global pixel, set when a sample observes it.
// other (may be NULL): a second pixel per sample; -1 there flags the sample.
__global__ void k_mark_bits(const int* pix, long long n, int n_pix, unsigned* bits, const int* other) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int g = pix[t];
    if (g >= 0 && g < n_pix && (!other || other[t] >= 0)) atomicOr(bits + (g >> 5), 1u << (g & 31));
  }
}

// Exclusive prefix of popcounts over the bit words (single block of 1024).
__global__ void __launch_bounds__(1024) k_scan_words(const unsigned* bits, int n_words, int* prefix, int* total) {
  __shared__ int part[1024];
  const int tid = threadIdx.x;
  const int chunk = (n_words + 1023) / 1024;
  const int b = tid * chunk, e = min(n_words, b + chunk);
  int acc = 0;
  for (int w = b; w < e; ++w) acc += __popc(bits[w]);
  part[tid] = acc;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int v = tid >= off ? part[tid - off] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  int run = part[tid] - acc;
  for (int w = b; w < e; ++w) {
    prefix[w] = run;
    run += __popc(bits[w]);
  }
  if (tid == 1023) *total = part[1023];
}

// Sharded plans: samples per global pixel on this rank (summed across ranks
// before the observed set is formed).
__global__ void k_count_pix(const int* pix, long long n, int n_pix, int* counts) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int g = pix[t];
    if (g >= 0 && g < n_pix) atomicAdd(counts + g, 1);
  }
}

// Samples t < n-1 with pix_obs[t] = pix_obs[t+1] >= 0 (block sums, one atomic per block).
__global__ void __launch_bounds__(256) k_count_repeats(const int* pix_obs, long long n, unsigned long long* count) {
  __shared__ unsigned long long part[8];
  unsigned long long c = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t + 1 < n; t += (long long)gridDim.x * blockDim.x) {
    const int q = pix_obs[t];
    c += (q >= 0 && q == pix_obs[t + 1]) ? 1ull : 0ull;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += part[w];
    atomicAdd(count, b);
  }
}

// One bit per global pixel observed by some rank (one thread per 32-pixel word).
__global__ void k_bits_from_counts(const int* counts, int n_pix, unsigned* bits) {
  const int n_words = (n_pix + 31) / 32;
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < n_words; w += gridDim.x * blockDim.x) {
    unsigned b = 0;
    for (int k = 0; k < 32 && 32 * w + k < n_pix; ++k)
      if (counts[32 * w + k] > 0) b |= 1u << k;
    bits[w] = b;
  }
}

// ---------------------------------------------------------------- deterministic plans
// The samples of every observed row in ascending order (a compressed row
// index): counts, an exclusive scan, an unordered fill, then each row sorted.
__global__ void k_count_rows(const int* pix_obs, long long n, int* counts) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int p = pix_obs[t];
    if (p >= 0) atomicAdd(counts + p, 1);
  }
}

// ptr[i] = counts[0] + ... + counts[i-1] for i = 0 .. n (single block of 1024).
__global__ void __launch_bounds__(1024) k_scan_rows(const int* counts, int n, int* ptr) {
  __shared__ long long part[1024];
  const int tid = threadIdx.x;
  const int chunk = (n + 1023) / 1024;
  const int b = min(n, tid * chunk), e = min(n, b + chunk);
  long long acc = 0;
  for (int i = b; i < e; ++i) acc += counts[i];
  part[tid] = acc;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const long long v = tid >= off ? part[tid - off] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  long long run = part[tid] - acc;
  for (int i = b; i < e; ++i) {
    ptr[i] = (int)run;
    run += counts[i];
  }
  if (tid == 1023) ptr[n] = (int)part[1023];
}

__global__ void k_fill_rows(const int* pix_obs, long long n, int* cursor, int* idx) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int p = pix_obs[t];
    if (p >= 0) idx[atomicAdd(cursor + p, 1)] = (int)t;
  }
}

// Insertion sort of each row (the fill leaves rows nearly in order).
__global__ void k_sort_rows(const int* ptr, int n_rows, int* idx) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_rows; p += gridDim.x * blockDim.x) {
    const int b = ptr[p], e = ptr[p + 1];
    for (int i = b + 1; i < e; ++i) {
      const int v = idx[i];
      int j = i - 1;
      while (j >= b && idx[j] > v) {
        idx[j + 1] = idx[j];
        --j;
      }
      idx[j + 1] = v;
    }
  }
}

__device__ __forceinline__ int rank_of(const unsigned* bits, const int* prefix, int g) {
  const unsigned w = bits[g >> 5];
  return prefix[g >> 5] + __popc(w & ((1u << (g & 31)) - 1u));
}

__global__ void k_obs2glob(const unsigned* bits, const int* prefix, int n_pix, int* obs2glob) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n_pix; g += gridDim.x * blockDim.x) {
    if (bits[g >> 5] & (1u << (g & 31))) obs2glob[rank_of(bits, prefix, g)] = g;
  }
}

__global__ void k_pix_obs(const int* pix, long long n, int n_pix, const unsigned* bits, const int* prefix,
                          int* pix_obs, const int* other) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int g = pix[t];
    pix_obs[t] = (g < 0 || g >= n_pix || (other && other[t] < 0)) ? -1 : rank_of(bits, prefix, g);
  }
}

// ---------------------------------------------------------------- compressed pointing
__global__ void k_validate_bore(const float4* bore, int n_bore, int* bad) {
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n_bore; u += gridDim.x * blockDim.x) {
    const float4 b = bore[u];
    if (!isfinite(b.x) || !isfinite(b.y) || !isfinite(b.z) || !isfinite(b.w)) atomicOr(bad, 8);
  }
}

// Section 5.4 bits for pointing expanded on the fly (Section 5.3).
__global__ void k_mark_bits_otf(const float4* bore, const StepDiv step, const float4* det, int n_per_det, long long n,
                                int W, int H, bool pol, unsigned* bits) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int dd = (int)(t / n_per_det);
    float c2, s2;
    const int g = expand_pointing(bore, step, (int)(t - (long long)dd * n_per_det), det[dd], W, H, pol, c2, s2);
    if (g >= 0) atomicOr(bits + (g >> 5), 1u << (g & 31));
  }
}

// observed row of every global pixel (-1: not observed)
__global__ void k_g2o(const unsigned* bits, const int* prefix, int n_pix, int* g2o) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n_pix; g += gridDim.x * blockDim.x)
    g2o[g] = (bits[g >> 5] & (1u << (g & 31))) ? rank_of(bits, prefix, g) : -1;
}

// the expanded pointing of every sample (global pixel and weights)
__global__ void k_expand_all(const float4* bore, const StepDiv step, const float4* det, int n_per_det, long long n,
                             int W, int H, bool pol, int* pix, float* c2o, float* s2o) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int dd = (int)(t / n_per_det);
    float c2, s2;
    const int g = expand_pointing(bore, step, (int)(t - (long long)dd * n_per_det), det[dd], W, H, pol, c2, s2);
    if (pix) pix[t] = g;
    if (c2o) c2o[t] = c2;
    if (s2o) s2o[t] = s2;
  }
}

// rows of excised pixels become zero (Section 4, gap filling)
__global__ void k_excise_g2o(const int* obs2glob, const unsigned char* excised, int n_obs, int* g2o) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_obs; k += gridDim.x * blockDim.x)
    if (excised[k]) g2o[obs2glob[k]] = -1;
}

__device__ __forceinline__ int interval_of(const long long* off, int n_ivl, long long t) {
  int lo = 0, hi = n_ivl;  // find i with off[i] <= t < off[i+1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= t) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Per-pixel sums for the preconditioner (Section 5): hits, A^T A and
// A^T W^-1 A with W^-1 = diag(N^-1), i.e. each sample weighted by f(0) of its
// interval's filter.  Also stores (cos 2psi, sin 2psi) in float64 for the FP64
// operator.  acc layout per pixel: T: [wsum]; IQU: [6 AtA | 6 AtWA].
// One pass over the samples: hit counts, and either the per-filter sums of
// w w^T of every pixel (G[filter][pixel][6], or [filter][pixel] for T) or
// directly A^T A and A^T W^-1 A (acc).  The first pass also stores the
// float64 and double-float weights; later passes read them back.
// Compressed pointing (ob.bore != NULL): pixel and weights expanded from the
// boresight nodes, the observed row looked up in g2o.

__global__ void k_accumulate(const int* pix_obs, const float* psi, long long n, const long long* off, int n_ivl,
                             const int* ivl_filter, const double* f0, int ns, double* acc, int* hits,
                             double2* cs64, float4* csdf, double* G, int n_obs, int first, const OtfPointing ob) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double c = 1.0, s = 0.0;
    int p;
    if (ob.bore) {
      float c2, s2;
      p = otf_row(ob, t, ns == 3, c2, s2);
      c = c2;
      s = s2;
    } else if (ns == 3) {
      if (first) {
        sincos(2.0 * (double)psi[t], &s, &c);
        cs64[t] = make_double2(c, s);
        const df64 cd(c), sd(s);
        csdf[t] = make_float4(cd.hi, cd.lo, sd.hi, sd.lo);
      } else {
        const double2 cs = cs64[t];
        c = cs.x;
        s = cs.y;
      }
    }
    if (!ob.bore) p = pix_obs[t];
    if (p < 0) continue;
    const int f = ivl_filter[interval_of(off, n_ivl, t)];
    atomicAdd(hits + p, 1);
    if (G) {
      if (ns == 1) {
        atomicAdd(G + (long long)f * n_obs + p, 1.0);
      } else {
        double* g = G + ((long long)f * n_obs + p) * 6;
        const double v[6] = {1.0, c, s, c * c, c * s, s * s};
#pragma unroll
        for (int k = 0; k < 6; ++k) atomicAdd(g + k, v[k]);
      }
      continue;
    }
    const double w0 = f0[f];
    if (ns == 1) {
      atomicAdd(acc + p, w0);
    } else {
      double* a = acc + 12LL * p;
      const double v[6] = {1.0, c, s, c * c, c * s, s * s};
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        atomicAdd(a + k, v[k]);
        atomicAdd(a + 6 + k, w0 * v[k]);
      }
    }
  }
}

// A^T A = sum_k G_k and A^T W^-1 A = sum_k f_k(0) G_k per pixel (the layout
// k_classify reads), in a fixed order over the filters.
__global__ void k_combine(const double* G, int n_filters, int n_obs, int ns, const double* f0, double* acc) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_obs; p += gridDim.x * blockDim.x) {
    if (ns == 1) {
      double sw = 0.0;
      for (int f = 0; f < n_filters; ++f) sw += f0[f] * G[(long long)f * n_obs + p];
      acc[p] = sw;
      continue;
    }
    for (int k = 0; k < 6; ++k) {
      double a = 0.0, aw = 0.0;
      for (int f = 0; f < n_filters; ++f) {
        const double g = G[((long long)f * n_obs + p) * 6 + k];
        a += g;
        aw += f0[f] * g;
      }
      acc[12LL * p + k] = a;
      acc[12LL * p + 6 + k] = aw;
    }
  }
}

// Eigenvalues of a symmetric 3x3 matrix by the trigonometric closed form
// (O. K. Smith, "Eigenvalues of a symmetric 3x3 matrix", CACM 4, 1961).
__device__ void sym3_eig(double a00, double a01, double a02, double a11, double a12, double a22, double& lmin,
                         double& lmax) {
  const double p1 = a01 * a01 + a02 * a02 + a12 * a12;
  if (p1 == 0.0) {
    lmin = fmin(a00, fmin(a11, a22));
    lmax = fmax(a00, fmax(a11, a22));
    return;
  }
  const double q = (a00 + a11 + a22) / 3.0;
  const double b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
  const double p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.0 * p1;
  const double p = sqrt(p2 / 6.0);
  const double ip = 1.0 / p;
  const double c00 = b00 * ip, c11 = b11 * ip, c22 = b22 * ip, c01 = a01 * ip, c02 = a02 * ip, c12 = a12 * ip;
  const double det = c00 * (c11 * c22 - c12 * c12) - c01 * (c01 * c22 - c12 * c02) + c02 * (c01 * c12 - c11 * c02);
  double r = 0.5 * det;
  r = fmin(1.0, fmax(-1.0, r));
  const double phi = acos(r) / 3.0;
  lmax = q + 2.0 * p * cos(phi);
  lmin = q + 2.0 * p * cos(phi + 2.0 * M_PI / 3.0);
}

// Classify observed pixels (IQU: excise when hits < 3 or rcond(A^T A) is
// below rcond_excise; flag float64 blocks below rcond_fp64) and invert the
// (A^T W^-1 A) blocks in float64.
__global__ void k_classify(const double* acc, const int* hits, int n_obs, int ns, double rc_ex, double rc_64,
                           double* P64, float* P32, unsigned char* excised, unsigned char* fp64flag, int* counts) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_obs; p += gridDim.x * blockDim.x) {
    if (ns == 1) {
      const bool ex = hits[p] == 0 || !(acc[p] > 0.0);
      const double inv = ex ? 0.0 : 1.0 / acc[p];
      P64[p] = inv;
      P32[p] = (float)inv;
      excised[p] = ex;
      fp64flag[p] = 0;
      if (ex) atomicAdd(counts, 1);
      continue;
    }
    const double* a = acc + 12LL * p;
    double lmin = 0.0, lmax = 0.0;
    sym3_eig(a[0], a[1], a[2], a[3], a[4], a[5], lmin, lmax);
    const double rc = lmax > 0.0 ? lmin / lmax : 0.0;
    bool ex = hits[p] < 3 || !(rc >= rc_ex);
    // inverse of the weighted block by cofactors
    const double m00 = a[6], m01 = a[7], m02 = a[8], m11 = a[9], m12 = a[10], m22 = a[11];
    const double A00 = m11 * m22 - m12 * m12, A01 = m02 * m12 - m01 * m22, A02 = m01 * m12 - m02 * m11;
    const double A11 = m00 * m22 - m02 * m02, A12 = m01 * m02 - m00 * m12, A22 = m00 * m11 - m01 * m01;
    const double det = m00 * A00 + m01 * A01 + m02 * A02;
    if (!(det > 0.0)) ex = true;
    const double id = ex ? 0.0 : 1.0 / det;
    const double inv[6] = {A00 * id, A01 * id, A02 * id, A11 * id, A12 * id, A22 * id};
    for (int k = 0; k < 6; ++k) {
      P64[6LL * p + k] = inv[k];
      P32[8LL * p + k] = (float)inv[k];
    }
    P32[8LL * p + 6] = 0.f;
    P32[8LL * p + 7] = 0.f;
    excised[p] = ex;
    const bool f64 = !ex && rc < rc_64;
    fp64flag[p] = f64;
    if (ex) atomicAdd(counts, 1);
    if (f64) atomicAdd(counts + 1, 1);
  }
}

// (pixel, angle) pairs read with one 8-byte load by the float32 operator
__global__ void k_pack_pw(const int* pix_obs, const float* psi, long long n, int2* pw) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    pw[t] = make_int2(pix_obs[t], __float_as_int(psi[t]));
}

// Rows of A observing excised pixels become zero (Section 4, gap filling).
__global__ void k_zero_excised_rows(int* pix_obs, long long n, const unsigned char* excised) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int p = pix_obs[t];
    if (p >= 0 && excised[p]) pix_obs[t] = -1;
  }
}

// ---------------------------------------------------------------- extended pointing
__global__ void k_ext_rows(const int* extra_index, long long n, int n_sky, int* ext_row) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int e = extra_index[t];
    ext_row[t] = e >= 0 ? n_sky + e : -1;
  }
}

// first half-wave-plate row of each sample's group (-1: none)
__global__ void k_hwp_base(const long long* off, int n_ivl, const int* ivl_base, long long n, int* base) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    base[t] = ivl_base[interval_of(off, n_ivl, t)];
}

__global__ void k_validate_hwp(const float* ang, const float* tau, long long n, int* bad) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    if (!isfinite(ang[t]) || !isfinite(tau[t])) atomicOr(bad, 32);
}

// Half-wave-plate parameters: sum over the surviving samples of f(0) C_{t,i}^2
// (the scalar preconditioner of each parameter).
__global__ void k_accumulate_hwp(const int* pix_obs, const int* hwp_base, const float* ang, const float* tau,
                                 long long n, const long long* off, int n_ivl, const int* ivl_filter, const double* f0,
                                 int row0, double* acc) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int b = hwp_base[t];
    if (b < 0 || pix_obs[t] < 0) continue;
    const double w0 = f0[ivl_filter[interval_of(off, n_ivl, t)]];
    double C[32];
    hwp_columns<double>(ang[t], tau[t], C);
#pragma unroll
    for (int i = 0; i < 32; ++i) atomic_add_warp(acc, (long long)(b - row0 + i), w0 * C[i] * C[i]);
  }
}

// Extra columns' sums over the samples whose row survives (sky pixel observed
// and not excised): hits and B^T W^-1 B (= sum of f(0)).
__global__ void k_accumulate_ext(const int* pix_obs, const int* ext_row, long long n, const long long* off, int n_ivl,
                                 const int* ivl_filter, const double* f0, int n_sky, int* hits, double* acc) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int r = ext_row[t];
    if (r < 0 || pix_obs[t] < 0) continue;
    atomicAdd(hits + (r - n_sky), 1);
    atomicAdd(acc + (r - n_sky), f0[ivl_filter[interval_of(off, n_ivl, t)]]);
  }
}

// Scalar blocks of the extra rows (slot 0; the rest of the row's block is 0).
// hits == NULL: half-wave-plate rows (excised when the weight sum is 0).
__global__ void k_classify_ext(const double* acc, const int* hits, int n_extra, int n_sky, int ns, double* P64,
                               float* P32, unsigned char* excised, unsigned char* fp64flag, int* counts) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_extra; e += gridDim.x * blockDim.x) {
    const long long r = n_sky + e;
    const bool ex = (hits && hits[e] == 0) || !(acc[e] > 0.0);
    const double inv = ex ? 0.0 : 1.0 / acc[e];
    if (ns == 1) {
      P64[r] = inv;
      P32[r] = (float)inv;
    } else {
      for (int k = 0; k < 6; ++k) P64[6 * r + k] = k == 0 ? inv : 0.0;
      for (int k = 0; k < 8; ++k) P32[8 * r + k] = k == 0 ? (float)inv : 0.f;
    }
    excised[r] = ex;
    fp64flag[r] = 0;
    if (ex) atomicAdd(counts, 1);
  }
}

// ---------------------------------------------------------------- multi-resolution preconditioner
// Section 6 with the block diagonal of Section 5 on each pixelisation: a 2 x 2
// (Q, U) block per polarisation pixel and a 1 x 1 block per intensity pixel;
// the I-QU couplings join different pixels and are left out.
// Polarisation sums per slot: hits, [cc cs ss] of A^T A and of A^T W^-1 A.
__global__ void k_accumulate_pol(const int* pix_pol, const float* psi, long long n, const long long* off, int n_ivl,
                                 const int* ivl_filter, const double* f0, double* acc, int* hits, double2* cs64,
                                 float4* csdf, int first) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double c, s;
    if (first) {
      sincos(2.0 * (double)psi[t], &s, &c);
      cs64[t] = make_double2(c, s);
      const df64 cd(c), sd(s);
      csdf[t] = make_float4(cd.hi, cd.lo, sd.hi, sd.lo);
    } else {
      const double2 cs = cs64[t];
      c = cs.x;
      s = cs.y;
    }
    const int q = pix_pol[t];
    if (q < 0) continue;
    const double w0 = f0[ivl_filter[interval_of(off, n_ivl, t)]];
    atomicAdd(hits + q, 1);
    double* a = acc + 6LL * q;
    const double v[3] = {c * c, c * s, s * s};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      atomicAdd(a + k, v[k]);
      atomicAdd(a + 3 + k, w0 * v[k]);
    }
  }
}

// Q/U blocks: excise below 2 hits or rcond(A^T A) < rc_ex (and slots past the
// observed count), flag float64 blocks below rc_64, invert the weighted 2 x 2
// block into entries (1,1), (1,2), (2,2) of the slot's 3 x 3 block.
__global__ void k_classify_pol(const double* acc, const int* hits, int n_slots, int n_obs_pol, double rc_ex,
                               double rc_64, double* P64, float* P32, unsigned char* excised_pol,
                               unsigned char* fp64flag, int* counts) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_slots; k += gridDim.x * blockDim.x) {
    bool ex = k >= n_obs_pol || hits[k] < 2;
    double rc = 0.0, i11 = 0.0, i12 = 0.0, i22 = 0.0;
    if (!ex) {
      const double* a = acc + 6LL * k;
      const double h = 0.5 * (a[0] + a[2]), d = 0.5 * (a[0] - a[2]);
      const double r = sqrt(d * d + a[1] * a[1]);
      const double lmax = h + r;
      // smaller eigenvalue as det / lmax (no cancellation when the block is near-singular)
      const double lmin = lmax > 0.0 ? (a[0] * a[2] - a[1] * a[1]) / lmax : 0.0;
      rc = lmax > 0.0 ? lmin / lmax : 0.0;
      ex = !(rc >= rc_ex);
      const double det = a[3] * a[5] - a[4] * a[4];
      if (!(det > 0.0)) ex = true;
      if (!ex) {
        const double id = 1.0 / det;
        i11 = a[5] * id;
        i12 = -a[4] * id;
        i22 = a[3] * id;
      }
    }
    const double v[6] = {0.0, 0.0, 0.0, i11, i12, i22};
    for (int j = 1; j < 6; ++j) {
      P64[6LL * k + j] = v[j];
      P32[8LL * k + j] = (float)v[j];
    }
    P32[8LL * k + 6] = 0.f;
    P32[8LL * k + 7] = 0.f;
    excised_pol[k] = ex;
    const bool f64 = !ex && rc < rc_64;
    fp64flag[k] = f64;
    if (ex && k < n_obs_pol) atomicAdd(counts + 1, 1);
    if (f64) atomicAdd(counts + 2, 1);
  }
}

// Rows whose polarisation pixel is excised become zero in both pixelisations.
__global__ void k_drop_rows_pol(int* pix, int* pix_pol, long long n, const unsigned char* excised_pol) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int q = pix_pol[t];
    if (q >= 0 && excised_pol[q]) {
      pix[t] = -1;
      pix_pol[t] = -1;
    }
  }
}

// Intensity sums from the remaining rows: hits and A^T W^-1 A (= sum of f(0)).
__global__ void k_accumulate_int(const int* pix, long long n, const long long* off, int n_ivl, const int* ivl_filter,
                                 const double* f0, double* acc, int* hits) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int p = pix[t];
    if (p < 0) continue;
    atomicAdd(hits + p, 1);
    atomicAdd(acc + p, f0[ivl_filter[interval_of(off, n_ivl, t)]]);
  }
}

// Intensity blocks: an I pixel without rows (or a slot past the count) is excised.
__global__ void k_classify_int(const double* acc, const int* hits, int n_slots, int n_obs_i, double* P64, float* P32,
                               unsigned char* excised, int* counts) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_slots; k += gridDim.x * blockDim.x) {
    const bool ex = k >= n_obs_i || hits[k] == 0 || !(acc[k] > 0.0);
    const double inv = ex ? 0.0 : 1.0 / acc[k];
    P64[6LL * k] = inv;
    P32[8LL * k] = (float)inv;
    excised[k] = ex;
    if (ex && k < n_obs_i) atomicAdd(counts, 1);
  }
}

static int grid_for(long long n, int threads = 256) {
  long long g = (n + threads - 1) / threads;
  if (g > 152LL * 32) g = 152LL * 32;
  if (g < 1) g = 1;
  return (int)g;
}

// ---------------------------------------------------------------- windows and tiles
struct Seg {
  long long ws, lo, hi;
  int out_lo, out_hi, filter;
};

static void make_segments(const std::vector<long long>& off, const std::vector<int>& filt, int n_lags, int M,
                          std::vector<Seg>& segs) {
  segs.clear();
  const long long h = n_lags - 1;
  const long long U = M - 2 * h;
  for (size_t i = 0; i + 1 < off.size(); ++i) {
    const long long t0 = off[i], t1 = off[i + 1], n = t1 - t0;
    if (n <= 0) continue;
    if (n + h <= M) {
      segs.push_back({t0, t0, t1, 0, (int)n, filt[i]});
      continue;
    }
    for (long long u0 = t0; u0 < t1; u0 += U) {
      const long long u1 = std::min(t1, u0 + U);
      const long long ws = u0 - h;
      segs.push_back({ws, std::max(t0, ws), std::min(t1, ws + M), (int)h, (int)(h + u1 - u0), filt[i]});
    }
  }
}

static void pair_tiles(const std::vector<Seg>& segs, int n_filters, std::vector<Tile>& tiles) {
  tiles.clear();
  for (int f = 0; f < n_filters; ++f) {
    std::vector<const Seg*> mine;
    for (const Seg& s : segs)
      if (s.filter == f) mine.push_back(&s);
    for (size_t k = 0; k < mine.size(); k += 2) {
      Tile T;
      memset(&T, 0, sizeof(T));
      T.filter = f;
      for (int l = 0; l < 2; ++l) {
        Lane& L = T.l[l];
        if (k + l < mine.size()) {
          const Seg* s = mine[k + l];
          L.ws = s->ws;
          L.lo = s->lo;
          L.hi = s->hi;
          L.out_lo = s->out_lo;
          L.out_hi = s->out_hi;
        } else {
          L.ws = 0;
          L.lo = 0;
          L.hi = 0;
          L.out_lo = 0;
          L.out_hi = 0;
        }
        L.rhs = 0;
      }
      tiles.push_back(T);
    }
  }
}

// Overlap-save windows of every interval, paired two per complex FFT
// (used by the allocation-free weighting entry point).
void build_tiles(const std::vector<long long>& off, const std::vector<int>& filt, int n_filters, int n_lags, int M,
                 std::vector<Tile>& tiles) {
  std::vector<Seg> segs;
  make_segments(off, filt, n_lags, M, segs);
  pair_tiles(segs, n_filters, tiles);
}

// Tile set for n_rhs right-hand sides sharing the pointing: lanes are
// (window, rhs) ordered by filter, window, rhs and paired consecutively, so
// right-hand sides 2j and 2j+1 of one window share a complex FFT and the
// pointing loads of the gather and scatter.
madmap_status ensure_wtod(Plan* p, int n_rhs) {
  if (!p->det || p->wtod_rhs >= n_rhs) return MADMAP_OK;
  void* buf = nullptr;
  madmap_status st = dalloc(p, &buf, sizeof(double) * (size_t)n_rhs * (size_t)std::max(1LL, p->n_t));
  if (st != MADMAP_OK) return st;
  p->wtod = buf;  // a smaller buffer stays with the plan until it is destroyed
  p->wtod_rhs = n_rhs;
  return MADMAP_OK;
}

static madmap_status build_det_rows(Plan* p, cudaStream_t s) {
  const long long n = p->n_t;
  int* counts = nullptr;
  madmap_status st = dalloc_t(p, &p->det_ptr, (size_t)p->n_obs + 1);
  if (st == MADMAP_OK) st = dalloc_t(p, &p->det_idx, (size_t)std::max(1LL, n));
  if (st != MADMAP_OK) return st;
  MM_CUDA(cudaMalloc(&counts, sizeof(int) * (size_t)std::max(1, p->n_obs)));
  cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)std::max(1, p->n_obs), s);
  if (n > 0) k_count_rows<<<grid_for(n), 256, 0, s>>>(p->pix_obs, n, counts);
  k_scan_rows<<<1, 1024, 0, s>>>(counts, p->n_obs, p->det_ptr);
  cudaMemcpyAsync(counts, p->det_ptr, sizeof(int) * (size_t)std::max(1, p->n_obs), cudaMemcpyDeviceToDevice, s);
  if (n > 0) k_fill_rows<<<grid_for(n), 256, 0, s>>>(p->pix_obs, n, counts, p->det_idx);
  if (p->n_obs > 0) k_sort_rows<<<grid_for(p->n_obs), 256, 0, s>>>(p->det_ptr, p->n_obs, p->det_idx);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaFree(counts);
  if (e != cudaSuccess) return cuda_fail(e, "deterministic row index");
  return ensure_wtod(p, 1);
}

madmap_status get_tile_set(Plan* p, int n_rhs, TileSet** out) {
  if (p->det) {
    madmap_status st = ensure_wtod(p, n_rhs);
    if (st != MADMAP_OK) return st;
  }
  for (TileSet* t : p->tile_sets)
    if (t->n_rhs == n_rhs) {
      *out = t;
      return MADMAP_OK;
    }
  std::vector<Seg> segs;
  make_segments(p->offsets, p->ivl_filter, p->n_lags, p->M, segs);
  std::vector<Tile> tiles;
  for (int f = 0; f < p->n_filters; ++f) {
    std::vector<std::pair<const Seg*, int>> lanes;
    for (const Seg& sg : segs)
      if (sg.filter == f)
        for (int r = 0; r < n_rhs; ++r) lanes.push_back({&sg, r});
    for (size_t k = 0; k < lanes.size(); k += 2) {
      Tile T;
      memset(&T, 0, sizeof(T));
      T.filter = f;
      for (int l = 0; l < 2; ++l) {
        Lane& L = T.l[l];
        if (k + l < lanes.size()) {
          const Seg* sg = lanes[k + l].first;
          L.ws = sg->ws;
          L.lo = sg->lo;
          L.hi = sg->hi;
          L.out_lo = sg->out_lo;
          L.out_hi = sg->out_hi;
          L.rhs = lanes[k + l].second;
        } else {
          L.rhs = lanes[k].second;  // empty lane: no input, no output
        }
      }
      tiles.push_back(T);
    }
  }
  TileSet* t = new TileSet();
  t->n_rhs = n_rhs;
  t->n_tiles = (int)tiles.size();
  madmap_status st = dalloc_t(p, &t->tiles, std::max<size_t>(1, tiles.size()));
  if (st != MADMAP_OK) {
    delete t;
    return st;
  }
  if (!tiles.empty()) {
    cudaError_t e = cudaMemcpy(t->tiles, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      delete t;
      return cuda_fail(e, "cudaMemcpy (tile set)");
    }
  }
  p->tile_sets.push_back(t);
  *out = t;
  return MADMAP_OK;
}

// Autotuning model for the FFT length: work ~ tiles * M * (log2 M + c), where
// c stands for the gather/scatter and memory passes per complex element.
static int choose_fft_len(const std::vector<long long>& off, const std::vector<int>& filt, int n_filters,
                          int n_lags) {
  double best = 1e300;
  int bestM = 0;
  std::vector<Seg> segs;
  std::vector<Tile> tiles;
  for (int lg = 8; lg <= 20; ++lg) {
    const int M = 1 << lg;
    if (M - 2 * (n_lags - 1) < 1) continue;
    make_segments(off, filt, n_lags, M, segs);
    pair_tiles(segs, n_filters, tiles);
    const double cost = (double)tiles.size() * (double)M * (lg + 8.0) + 1.0 * M;
    if (cost < best) {
      best = cost;
      bestM = M;
    }
  }
  return bestM;
}

// Spectrum of one filter's circulant embedding into h64/h32/hdf (the layout
// the row kernel reads); returns false when the symbol is not positive.
static bool filter_spectrum(const Plan* p, int f, double* h64, float* h32, df64* hdf, double* min_out) {
  const int M = p->M;
  std::vector<double> re(M, 0.0), im(M, 0.0);
  const double* lg = &p->lags[(size_t)f * p->n_lags];
  re[0] = lg[0];
  for (int t = 1; t < p->n_lags; ++t) {
    re[t] += lg[t];
    re[M - t] += lg[t];
  }
  host_fft(re, im, false);
  double mn = 1e300;
  for (int k = 0; k < M; ++k) mn = std::min(mn, re[k]);
  *min_out = mn;
  if (!(mn > 0.0)) return false;
  for (int pos2 = 0; pos2 < p->N2; ++pos2) {
    int k2 = 0;
    for (int b = 0; b < p->logN2; ++b) k2 |= ((pos2 >> b) & 1) << (p->logN2 - 1 - b);
    for (int pos1 = 0; pos1 < p->N1; ++pos1) {
      int k1 = 0;
      for (int b = 0; b < p->logN1; ++b) k1 |= ((pos1 >> b) & 1) << (p->logN1 - 1 - b);
      const double v = re[k2 + (size_t)p->N2 * k1] / (double)M;
      const size_t o = (size_t)pos2 * p->N1 + pos1;
      h64[o] = v;
      h32[o] = (float)v;
      hdf[o] = df64(v);
    }
  }
  return true;
}

// All filters' spectra, computed on host threads (one filter per task).
static madmap_status build_spectra(Plan* p) {
  const int M = p->M, F = p->n_filters;
  std::vector<double> h64((size_t)F * M);
  std::vector<float> h32((size_t)F * M);
  std::vector<df64> hdf((size_t)F * M);
  std::vector<double> mins(F, 0.0);
  std::vector<char> ok(F, 0);
  const int T = std::max(1, std::min<int>(F, (int)std::max(1u, std::thread::hardware_concurrency())));
  std::atomic<int> next(0);
  auto work = [&]() {
    for (int f = next++; f < F; f = next++)
      ok[f] = filter_spectrum(p, f, &h64[(size_t)f * M], &h32[(size_t)f * M], &hdf[(size_t)f * M], &mins[f]);
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < T; ++t) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
  for (int f = 0; f < F; ++f)
    if (!ok[f]) {
      set_error("filter " + std::to_string(f) + " is not positive definite (circulant symbol minimum " +
                std::to_string(mins[f]) + ")");
      return MADMAP_ERR_NOT_PD;
    }
  MM_CUDA(cudaMemcpy(p->H64, h64.data(), h64.size() * sizeof(double), cudaMemcpyHostToDevice));
  MM_CUDA(cudaMemcpy(p->H32, h32.data(), h32.size() * sizeof(float), cudaMemcpyHostToDevice));
  MM_CUDA(cudaMemcpy(p->Hdf, hdf.data(), hdf.size() * sizeof(df64), cudaMemcpyHostToDevice));
  return MADMAP_OK;
}

// Multi-resolution preconditioner and classification.  Every call passes over
// the samples (no per-filter sums are kept); the first also stores the
// float64 weights, zeroes the rows of excised Q/U pixels and packs the
// float32 pointing.  Later calls see the same rows, so the classification
// cannot change.
static madmap_status build_preconditioner_mr(Plan* p, cudaStream_t s) {
  const long long n = p->n_t;
  const int n_obs = p->n_obs;
  const bool first = !p->pre_built;
  if (first) {
    madmap_status a = dalloc_t(p, &p->hits, (size_t)std::max(1, n_obs));
    if (a != MADMAP_OK) return a;
  }
  const size_t ns1 = (size_t)std::max(1, n_obs);
  double *acc_pol = nullptr, *acc_i = nullptr, *df0 = nullptr;
  int *hits_pol = nullptr, *dfilt = nullptr, *counts = nullptr;
  long long* doff = nullptr;
  auto cleanup = [&]() {
    cudaFree(acc_pol);
    cudaFree(acc_i);
    cudaFree(df0);
    cudaFree(hits_pol);
    cudaFree(dfilt);
    cudaFree(counts);
    cudaFree(doff);
  };
  cudaError_t e = cudaSuccess;
  if ((e = cudaMalloc(&acc_pol, sizeof(double) * ns1 * 6)) != cudaSuccess ||
      (e = cudaMalloc(&acc_i, sizeof(double) * ns1)) != cudaSuccess ||
      (e = cudaMalloc(&hits_pol, sizeof(int) * ns1)) != cudaSuccess ||
      (e = cudaMalloc(&doff, sizeof(long long) * (p->n_ivl + 1))) != cudaSuccess ||
      (e = cudaMalloc(&dfilt, sizeof(int) * std::max(1, p->n_ivl))) != cudaSuccess ||
      (e = cudaMalloc(&df0, sizeof(double) * p->n_filters)) != cudaSuccess ||
      (e = cudaMalloc(&counts, sizeof(int) * 3)) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "cudaMalloc (preconditioner temporaries)");
  }
  std::vector<double> f0(p->n_filters);
  for (int f = 0; f < p->n_filters; ++f) f0[f] = p->lags[(size_t)f * p->n_lags];
  cudaMemsetAsync(acc_pol, 0, sizeof(double) * ns1 * 6, s);
  cudaMemsetAsync(acc_i, 0, sizeof(double) * ns1, s);
  cudaMemsetAsync(hits_pol, 0, sizeof(int) * ns1, s);
  cudaMemsetAsync(p->hits, 0, sizeof(int) * ns1, s);
  cudaMemsetAsync(counts, 0, sizeof(int) * 3, s);
  cudaMemcpyAsync(doff, p->offsets.data(), sizeof(long long) * (p->n_ivl + 1), cudaMemcpyHostToDevice, s);
  if (p->n_ivl) cudaMemcpyAsync(dfilt, p->ivl_filter.data(), sizeof(int) * p->n_ivl, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(df0, f0.data(), sizeof(double) * p->n_filters, cudaMemcpyHostToDevice, s);
  if (n > 0)
    k_accumulate_pol<<<grid_for(n), 256, 0, s>>>(p->pix_obs_pol, p->psi, n, doff, p->n_ivl, dfilt, df0, acc_pol,
                                                  hits_pol, p->cs64, p->csdf, first ? 1 : 0);
  if (n_obs > 0)
    k_classify_pol<<<grid_for(n_obs), 256, 0, s>>>(acc_pol, hits_pol, n_obs, p->n_obs_pol, p->rcond_excise,
                                                    p->rcond_fp64, p->P64, p->P32, p->excised_pol, p->fp64flag,
                                                    counts);
  if (first && n > 0) k_drop_rows_pol<<<grid_for(n), 256, 0, s>>>(p->pix_obs, p->pix_obs_pol, n, p->excised_pol);
  if (n > 0)
    k_accumulate_int<<<grid_for(n), 256, 0, s>>>(p->pix_obs, n, doff, p->n_ivl, dfilt, df0, acc_i, p->hits);
  if (n_obs > 0)
    k_classify_int<<<grid_for(n_obs), 256, 0, s>>>(acc_i, p->hits, n_obs, p->n_obs_i, p->P64, p->P32, p->excised,
                                                    counts);
  if (first && n > 0) k_pack_pw<<<grid_for(n), 256, 0, s>>>(p->pix_obs, p->psi, n, p->pw);
  int hc[3] = {0, 0, 0};
  e = cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  cleanup();
  if (e != cudaSuccess) return cuda_fail(e, "preconditioner build");
  p->n_excised = hc[0];
  p->n_excised_pol = hc[1];
  p->n_fp64 = hc[2];
  p->pre_built = true;
  return MADMAP_OK;
}

// Block preconditioner (A^T W^-1 A)^-1 and the pixel classification.  The
// first call passes over the samples; when the per-filter sums G fit in
// 512 MB they are kept, so a change of filters (set_filters) only recombines
// them per pixel with the new f(0) and reinverts the blocks.  The first
// call's hit counts are kept too, so the classification cannot change.
static madmap_status build_preconditioner(Plan* p, cudaStream_t s) {
  if (p->multires) return build_preconditioner_mr(p, s);
  const long long n = p->n_t;
  const int n_obs = p->ext ? p->n_obs_sky : p->n_obs;  // sky rows (extra rows follow)
  const int ns = p->n_stokes;
  const int nb = ns == 1 ? 1 : 6;
  const bool first = !p->pre_built;
  if (first) {
    madmap_status a = dalloc_t(p, &p->hits, (size_t)std::max(1, n_obs));
    if (a != MADMAP_OK) return a;
    const size_t gbytes = sizeof(double) * (size_t)p->n_filters * n_obs * nb;
    if (n_obs > 0 && gbytes <= ((size_t)512 << 20)) {
      a = dalloc(p, (void**)&p->G, gbytes);
      if (a != MADMAP_OK) return a;
    }
  }
  double* acc = nullptr;
  long long* doff = nullptr;
  int* dfilt = nullptr;
  double* df0 = nullptr;
  int* counts = nullptr;
  // temporaries (freed at the end)
  MM_CUDA(cudaMalloc(&acc, sizeof(double) * (size_t)std::max(1, n_obs) * (ns == 1 ? 1 : 12)));
  madmap_status st = MADMAP_OK;
  auto cleanup = [&]() {
    cudaFree(acc);
    cudaFree(doff);
    cudaFree(dfilt);
    cudaFree(df0);
    cudaFree(counts);
  };
  cudaError_t e = cudaSuccess;
  std::vector<double> f0(p->n_filters);
  for (int f = 0; f < p->n_filters; ++f) f0[f] = p->lags[(size_t)f * p->n_lags];
  if ((e = cudaMalloc(&doff, sizeof(long long) * (p->n_ivl + 1))) != cudaSuccess ||
      (e = cudaMalloc(&dfilt, sizeof(int) * std::max(1, p->n_ivl))) != cudaSuccess ||
      (e = cudaMalloc(&df0, sizeof(double) * p->n_filters)) != cudaSuccess ||
      (e = cudaMalloc(&counts, sizeof(int) * 4)) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "cudaMalloc (preconditioner temporaries)");
  }
  cudaMemsetAsync(acc, 0, sizeof(double) * (size_t)std::max(1, n_obs) * (ns == 1 ? 1 : 12), s);
  cudaMemsetAsync(counts, 0, sizeof(int) * 4, s);
  cudaMemcpyAsync(doff, p->offsets.data(), sizeof(long long) * (p->n_ivl + 1), cudaMemcpyHostToDevice, s);
  if (p->n_ivl) cudaMemcpyAsync(dfilt, p->ivl_filter.data(), sizeof(int) * p->n_ivl, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(df0, f0.data(), sizeof(double) * p->n_filters, cudaMemcpyHostToDevice, s);
  if (first || !p->G) {
    cudaMemsetAsync(p->hits, 0, sizeof(int) * (size_t)std::max(1, n_obs), s);
    if (p->G) cudaMemsetAsync(p->G, 0, sizeof(double) * (size_t)p->n_filters * n_obs * nb, s);
    if (n > 0)
      k_accumulate<<<grid_for(n), 256, 0, s>>>(p->pix_obs, p->psi, n, doff, p->n_ivl, dfilt, df0, ns, acc, p->hits,
                                                p->cs64, p->csdf, p->G, n_obs, first ? 1 : 0, otf_pointing(p));
  }
  if (p->G && n_obs > 0)
    k_combine<<<grid_for(n_obs), 256, 0, s>>>(p->G, p->n_filters, n_obs, ns, df0, acc);
  if (p->allreduce && n_obs > 0) {
    // sharded plans: the blocks and hit counts of all ranks (hits only when
    // they were accumulated anew: a kept per-filter sum reuses the global ones)
    st = reduce_across(p, acc, (long long)n_obs * (ns == 1 ? 1 : 12), MADMAP_REDUCE_F64, s);
    if (st == MADMAP_OK && (first || !p->G)) st = reduce_across(p, p->hits, n_obs, MADMAP_REDUCE_I32, s);
    if (st != MADMAP_OK) {
      cleanup();
      return st;
    }
  }
  if (n_obs > 0)
    k_classify<<<grid_for(n_obs), 256, 0, s>>>(acc, p->hits, n_obs, ns, p->rcond_excise, p->rcond_fp64, p->P64,
                                                p->P32, p->excised, p->fp64flag, counts);
  if (p->otf) {
    if (first && n_obs > 0) k_excise_g2o<<<grid_for(n_obs), 256, 0, s>>>(p->obs2glob, p->excised, n_obs, p->g2o);
  } else {
    if (first && n > 0) k_zero_excised_rows<<<grid_for(n), 256, 0, s>>>(p->pix_obs, n, p->excised);
    if (first && n > 0 && ns == 3) k_pack_pw<<<grid_for(n), 256, 0, s>>>(p->pix_obs, p->psi, n, p->pw);
  }
  int* hits_e = nullptr;
  double* acc_e = nullptr;
  if (p->n_extra > 0) {  // the extra columns, from the rows that survive the sky's excision
    if ((e = cudaMalloc(&hits_e, sizeof(int) * p->n_extra)) != cudaSuccess ||
        (e = cudaMalloc(&acc_e, sizeof(double) * p->n_extra)) != cudaSuccess) {
      cudaFree(hits_e);
      cudaFree(acc_e);
      cleanup();
      return cuda_fail(e, "cudaMalloc (preconditioner temporaries)");
    }
    cudaMemsetAsync(hits_e, 0, sizeof(int) * p->n_extra, s);
    cudaMemsetAsync(acc_e, 0, sizeof(double) * p->n_extra, s);
    if (n > 0)
      k_accumulate_ext<<<grid_for(n), 256, 0, s>>>(p->pix_obs, p->ext_row, n, doff, p->n_ivl, dfilt, df0, n_obs,
                                                    hits_e, acc_e);
    if (p->n_extra > 0)
      k_classify_ext<<<grid_for(p->n_extra), 256, 0, s>>>(acc_e, hits_e, p->n_extra, n_obs, ns, p->P64, p->P32,
                                                           p->excised, p->fp64flag, counts + 2);
  }
  double* acc_h = nullptr;
  const int n_hwp = 32 * p->n_hwp_groups;
  if (n_hwp > 0) {
    if ((e = cudaMalloc(&acc_h, sizeof(double) * n_hwp)) != cudaSuccess) {
      cudaFree(hits_e);
      cudaFree(acc_e);
      cleanup();
      return cuda_fail(e, "cudaMalloc (preconditioner temporaries)");
    }
    cudaMemsetAsync(acc_h, 0, sizeof(double) * n_hwp, s);
    if (n > 0)
      k_accumulate_hwp<<<grid_for(n), 256, 0, s>>>(p->pix_obs, p->hwp_base, p->hwp_ang, p->hwp_tau, n, doff, p->n_ivl,
                                                    dfilt, df0, p->hwp_row0, acc_h);
    k_classify_ext<<<grid_for(n_hwp), 256, 0, s>>>(acc_h, nullptr, n_hwp, p->hwp_row0, ns, p->P64, p->P32,
                                                    p->excised, p->fp64flag, counts + 3);
  }
  int hc[4] = {0, 0, 0, 0};
  e = cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaFree(hits_e);
  cudaFree(acc_e);
  cudaFree(acc_h);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(e, "preconditioner build");
  p->n_excised = hc[0];
  p->n_fp64 = hc[1];
  p->n_excised_extra = hc[2];
  p->n_excised_hwp = hc[3];
  p->pre_built = true;
  return st;
}

madmap_status reduce_across(Plan* p, void* buf, long long count, int dtype, cudaStream_t s) {
  if (!p->allreduce || count <= 0) return MADMAP_OK;
  MM_CUDA(cudaGetLastError());
  const int32_t rc = p->allreduce(buf, (int64_t)count, dtype, static_cast<void*>(s), p->allreduce_user);
  MM_CHECK(rc == 0, MADMAP_ERR_INTERNAL, "the allreduce callback of a sharded plan failed");
  return MADMAP_OK;
}

// Windows, spectra, twiddles, chunking, streams and scratch for FFT length M
// (replacing those of an earlier length).  tpc_req > 0 fixes the tiles per
// launch chunk.
static madmap_status setup_windows(Plan* p, int M, long long tpc_req, cudaStream_t s) {
  free_windows(p);
  p->M = M;
  {
    // column transforms of 2^ceil(lg/2) points, or half that when the
    // autotuner found the shorter columns faster
    const int lg = ilog2((unsigned)p->M);
    p->logN2 = (lg + 1) / 2 - p->split_down;
    p->logN1 = lg - p->logN2;
    if (p->logN2 < 1 || p->logN1 > 10) {
      set_error("fft_split: the row transforms would exceed 1024 points");
      return MADMAP_ERR_INVALID_ARG;
    }
    p->N1 = 1 << p->logN1;
    p->N2 = 1 << p->logN2;
  }
  std::vector<Seg> segs;
  make_segments(p->offsets, p->ivl_filter, p->n_lags, p->M, segs);
  p->host_tiles.clear();
  pair_tiles(segs, p->n_filters, p->host_tiles);
  p->n_segments = (int)segs.size();
  p->n_tiles = (int)p->host_tiles.size();
  {
    // Chunk size: launches of many CTA waves let CTAs in different phases
    // (gather, FFT passes, scatter) overlap on each SM, which beat wave-sized
    // chunks whose scratch stays in L2.  At most 1 GB of scratch per chunk
    // (float64 sizing), and at least two chunks when there are 16 tiles or
    // more: chunks alternate between two streams, so each launch's tail
    // overlaps the next chunk (4 x 2^22-sample IQU scan: 0.325 ms against 0.341 ms in one launch).
    long long tpc = tpc_req;
    if (tpc <= 0) {
      tpc = std::max(1LL, (1LL << 30) / (16LL * p->M));
      if (p->n_tiles >= 16) tpc = std::min<long long>(tpc, (p->n_tiles + 1) / 2);
    }
    tpc = std::max(1LL, std::min<long long>(tpc, std::max(1, p->n_tiles)));
    tpc = std::min<long long>(tpc, 65535);
    p->tiles_per_chunk = (int)tpc;
  }
  madmap_status st = walloc_t(p, &p->tiles, std::max(1, p->n_tiles));
  if (st != MADMAP_OK) return st;
  if (p->n_tiles)
    MM_CUDA(cudaMemcpy(p->tiles, p->host_tiles.data(), sizeof(Tile) * p->n_tiles, cudaMemcpyHostToDevice));
  if ((st = walloc_t(p, &p->H64, (size_t)p->n_filters * p->M)) != MADMAP_OK) return st;
  if ((st = walloc_t(p, &p->H32, (size_t)p->n_filters * p->M)) != MADMAP_OK) return st;
  if ((st = walloc_t(p, &p->Hdf, (size_t)p->n_filters * p->M)) != MADMAP_OK) return st;
  if ((st = build_spectra(p)) != MADMAP_OK) return st;
  {
    std::vector<double2> t64(p->M);
    std::vector<float2> t32(p->M);
    std::vector<cdf64> tdf(p->M);
    for (int j = 0; j < p->M; ++j) {
      const double ang = 2.0 * M_PI * (double)j / (double)p->M;
      t64[j] = make_double2(cos(ang), -sin(ang));
      t32[j] = make_float2((float)t64[j].x, (float)t64[j].y);
      tdf[j].x = df64(t64[j].x);
      tdf[j].y = df64(t64[j].y);
    }
    if ((st = walloc_t(p, &p->tw64, p->M)) != MADMAP_OK) return st;
    if ((st = walloc_t(p, &p->tw32, p->M)) != MADMAP_OK) return st;
    if ((st = walloc_t(p, &p->twdf, p->M)) != MADMAP_OK) return st;
    MM_CUDA(cudaMemcpy(p->tw64, t64.data(), sizeof(double2) * p->M, cudaMemcpyHostToDevice));
    MM_CUDA(cudaMemcpy(p->tw32, t32.data(), sizeof(float2) * p->M, cudaMemcpyHostToDevice));
    MM_CUDA(cudaMemcpy(p->twdf, tdf.data(), sizeof(cdf64) * p->M, cudaMemcpyHostToDevice));
  }
  {
    const int n_chunks = p->n_tiles ? (p->n_tiles + p->tiles_per_chunk - 1) / p->tiles_per_chunk : 0;
    p->scratch_slots = n_chunks > 1 ? 2 : 1;
    if (n_chunks > 1 && !p->op_stream[0]) {
      for (int i = 0; i < 2; ++i) {
        MM_CUDA(cudaStreamCreateWithFlags(&p->op_stream[i], cudaStreamNonBlocking));
        MM_CUDA(cudaEventCreateWithFlags(&p->op_join[i], cudaEventDisableTiming));
      }
      MM_CUDA(cudaEventCreateWithFlags(&p->op_fork, cudaEventDisableTiming));
    }
  }
  return walloc(p, &p->scratch, (size_t)p->scratch_slots * p->tiles_per_chunk * p->M * sizeof(double2));
}

// Plans whose column kernels can sum runs of one pixel before the scatter's
// atomics (stored temperature or IQU pointing, one pixelisation, no extra
// columns, map sums by atomics).
static bool runs_capable(const Plan* p) {
  return !p->otf && !p->multires && !p->ext && !p->det && !p->diag && (p->n_stokes == 1 || p->n_stokes == 3);
}
// the fraction of repeated samples from which run sums are the default
static constexpr double kRunsMinFrac = 0.25;

// Measuring autotuner: time the float32 operator (CUDA events on `s`, after a
// warm-up application) for every candidate FFT length (the given one, or the
// cost model's choice and its neighbours a factor two either way) and tiles
// per launch chunk (the given number, or the default rule and half and twice
// it); at the fastest of those, the other split of the length into column and
// row transforms (columns half as long, rows twice) and then the scatter with
// and without run sums.  The fastest candidate is kept; all of them are
// reported in the plan's stats.
static madmap_status autotune_windows(Plan* p, int M_fixed, int M0, long long tpc_fixed, cudaStream_t s) {
  std::vector<int> Ms;
  for (int M : {M0 / 2, M0, 2 * M0})
    if ((M_fixed == 0 || M == M_fixed) && M >= 256 && M <= (1 << 20) && M - 2 * (p->n_lags - 1) >= 1 &&
        ilog2((unsigned)M) - ((ilog2((unsigned)M) + 1) / 2 - p->split_down) <= 10)
      Ms.push_back(M);
  const long long nv = (long long)std::max(1, p->n_obs) * p->ns_pad;
  float *x = nullptr, *y = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    cudaFree(x);
    cudaFree(y);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  cudaError_t ce = cudaMalloc(&x, sizeof(float) * nv);
  if (ce == cudaSuccess) ce = cudaMalloc(&y, sizeof(float) * nv);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(x, 0, sizeof(float) * nv, s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(y, 0, sizeof(float) * nv, s);
  if (ce != cudaSuccess) {
    cleanup();
    return cuda_fail(ce, "autotune buffers");
  }
  p->tuned.clear();
  int bestM = M0;
  long long bestT = tpc_fixed;
  float best = 3.4e38f;
  madmap_status st = MADMAP_OK;
  for (int M : Ms) {
    std::vector<long long> tpcs;
    if (tpc_fixed > 0) {
      tpcs.push_back(tpc_fixed);
    } else {
      if ((st = setup_windows(p, M, 0, s)) != MADMAP_OK) break;
      const long long t0 = p->tiles_per_chunk;
      for (long long t : {t0 / 2, t0, 2 * t0})
        if (t >= 1 && (t < 2 * t0 || t <= p->n_tiles) && std::find(tpcs.begin(), tpcs.end(), t) == tpcs.end())
          tpcs.push_back(t);
    }
    for (long long tpc : tpcs) {
      if ((st = setup_windows(p, M, tpc, s)) != MADMAP_OK) break;
      if ((st = op_launch(p, OPP_F32, IN_MAP, OUT_MAP, x, y, 0, 0, 1, nullptr, s)) != MADMAP_OK) break;
      const int reps = 3;
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps && st == MADMAP_OK; ++r)
        st = op_launch(p, OPP_F32, IN_MAP, OUT_MAP, x, y, 0, 0, 1, nullptr, s);
      cudaEventRecord(e1, s);
      if (st != MADMAP_OK) break;
      float ms = 0.f;
      if ((ce = cudaEventSynchronize(e1)) != cudaSuccess || (ce = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
        st = cuda_fail(ce, "autotune timing");
        break;
      }
      ms /= reps;
      p->tuned.push_back({M, (int)p->tiles_per_chunk, ms, p->runs, p->N2});
      if (ms < best) {
        best = ms;
        bestM = M;
        bestT = p->tiles_per_chunk;
      }
    }
    if (st != MADMAP_OK) break;
  }
  // one more candidate at the best geometry so far: one operator warm-up
  // application, then the mean of three
  auto time_current = [&](float* out_ms) -> madmap_status {
    madmap_status r = MADMAP_OK;
    for (int pass = 0; pass < 2 && r == MADMAP_OK; ++pass) {
      if (pass == 1) cudaEventRecord(e0, s);
      for (int k = 0; k < (pass ? 3 : 1) && r == MADMAP_OK; ++k)
        r = op_launch(p, OPP_F32, IN_MAP, OUT_MAP, x, y, 0, 0, 1, nullptr, s);
    }
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (r == MADMAP_OK &&
        ((ce = cudaEventSynchronize(e1)) != cudaSuccess || (ce = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess))
      r = cuda_fail(ce, "autotune timing");
    *out_ms = ms / 3;
    return r;
  };
  // the other split of the best length: columns of half the length (kept when
  // both transforms still have compile-time geometry)
  if (st == MADMAP_OK && !p->split_fixed) {
    const int lg = ilog2((unsigned)bestM), l2 = (lg + 1) / 2 - 1, l1 = lg - l2;
    if (l2 >= 7 && l2 <= 10 && l1 >= 6 && l1 <= 10) {
      p->split_down = 1;
      float ms = 0.f;
      if ((st = setup_windows(p, bestM, bestT, s)) == MADMAP_OK && (st = time_current(&ms)) == MADMAP_OK) {
        p->tuned.push_back({bestM, (int)p->tiles_per_chunk, ms, p->runs, p->N2});
        if (ms < best) best = ms;
        else p->split_down = 0;
      }
    }
  }
  // the other scatter mode at the best geometry
  if (st == MADMAP_OK && runs_capable(p) && !p->runs_fixed) {
    const int r0 = p->runs;
    st = setup_windows(p, bestM, bestT, s);
    p->runs = 1 - r0;
    float ms = 0.f;
    if (st == MADMAP_OK && (st = time_current(&ms)) == MADMAP_OK) {
      p->tuned.push_back({bestM, (int)p->tiles_per_chunk, ms, p->runs, p->N2});
      if (!(ms < best)) p->runs = r0;
    }
  }
  cleanup();
  if (st != MADMAP_OK) return st;
  return setup_windows(p, bestM, bestT, s);
}

}  // namespace mm

// ---------------------------------------------------------------- C ABI
extern "C" madmap_status madmap_partition_intervals(int32_t n_intervals, const int64_t* off, int32_t n_ranks,
                                                    int32_t* first) {
  using namespace mm;
  MM_CHECK(n_intervals >= 0 && n_ranks >= 1 && off && first, MADMAP_ERR_INVALID_ARG,
           "partition_intervals: bad arguments");
  MM_CHECK(off[0] == 0, MADMAP_ERR_INVALID_ARG, "partition_intervals: interval_offsets must start at 0");
  for (int i = 0; i < n_intervals; ++i)
    MM_CHECK(off[i + 1] >= off[i], MADMAP_ERR_INVALID_ARG, "partition_intervals: offsets must be non-decreasing");
  const long long total = off[n_intervals];
  first[0] = 0;
  int j = 0;
  for (int r = 0; r + 1 < n_ranks; ++r) {
    // the boundary nearest to the rank's share of the samples (ties: the earlier one)
    const long double target = (long double)total * (r + 1) / n_ranks;
    const int prev = j;
    while (j < n_intervals && (long double)off[j + 1] <= target) ++j;
    if (j < n_intervals && (long double)off[j + 1] - target < target - (long double)off[j]) ++j;
    while (j > prev && off[j - 1] == off[j]) --j;  // of equal boundaries (empty intervals), the earliest
    first[r + 1] = j;
  }
  first[n_ranks] = n_intervals;
  return MADMAP_OK;
}

extern "C" madmap_status madmap_plan_create(const madmap_plan_desc* d, void* stream, madmap_plan_t* out) {
  MM_CHECK(out != nullptr, MADMAP_ERR_INVALID_ARG, "plan_create: out is NULL");
  *out = nullptr;
  MM_CHECK(d != nullptr, MADMAP_ERR_INVALID_ARG, "plan_create: desc is NULL");
  MM_CHECK(d->n_stokes == 1 || d->n_stokes == 3, MADMAP_ERR_INVALID_ARG, "n_stokes must be 1 or 3");
  MM_CHECK(d->n_samples >= 0 && d->n_samples < (1LL << 40), MADMAP_ERR_INVALID_ARG, "bad n_samples");
  MM_CHECK(d->n_pix > 0, MADMAP_ERR_INVALID_ARG, "n_pix must be > 0");
  const bool otf = d->boresight != nullptr;
  if (otf) {
    MM_CHECK(!d->pix && !d->psi && !d->pix_pol, MADMAP_ERR_INVALID_ARG,
             "compressed pointing: pix, psi and pix_pol must be NULL");
    MM_CHECK(d->n_det >= 1 && d->det_pointing && d->n_samples % d->n_det == 0, MADMAP_ERR_INVALID_ARG,
             "compressed pointing: need n_det >= 1 dividing n_samples and det_pointing");
    MM_CHECK(d->n_samples / d->n_det < (1LL << 31) - 1, MADMAP_ERR_INVALID_ARG,
             "compressed pointing: too many samples per detector");
    MM_CHECK(d->bore_step >= 1, MADMAP_ERR_INVALID_ARG, "compressed pointing: bore_step must be >= 1");
    const long long npd = d->n_samples / d->n_det;
    MM_CHECK(npd == 0 || (long long)d->n_bore >= (npd - 1) / d->bore_step + 2, MADMAP_ERR_INVALID_ARG,
             "compressed pointing: n_bore must be >= (n_per_det - 1) / bore_step + 2");
    MM_CHECK(d->grid_width >= 1 && d->grid_height >= 1 && d->grid_width <= (1 << 24) &&
                 d->grid_height <= (1 << 24) && (long long)d->grid_width * d->grid_height == d->n_pix,
             MADMAP_ERR_INVALID_ARG, "compressed pointing: n_pix must equal grid_width * grid_height");
    for (int k = 0; k < 4 * d->n_det; ++k)
      MM_CHECK(isfinite(d->det_pointing[k]), MADMAP_ERR_INVALID_ARG, "compressed pointing: det_pointing not finite");
    for (int i = 0; i < d->n_intervals && npd > 0 && d->interval_offsets; ++i)
      MM_CHECK(d->interval_offsets[i + 1] <= d->interval_offsets[i] ||
                   d->interval_offsets[i] / npd == (d->interval_offsets[i + 1] - 1) / npd,
               MADMAP_ERR_INVALID_ARG, "compressed pointing: an interval spans two detectors");
  } else {
    MM_CHECK(d->n_samples == 0 || d->pix != nullptr, MADMAP_ERR_INVALID_ARG, "pix is NULL");
    MM_CHECK((d->n_stokes == 1) == (d->psi == nullptr) || d->n_samples == 0, MADMAP_ERR_INVALID_ARG,
             "psi must be NULL for T and non-NULL for IQU");
  }
  MM_CHECK(!d->pix_pol || (d->n_stokes == 3 && d->n_pix_pol > 0), MADMAP_ERR_INVALID_ARG,
           "pix_pol needs n_stokes = 3 and n_pix_pol > 0");
  MM_CHECK(!d->extra_index || (d->n_extra >= 1 && !d->pix_pol && !d->boresight), MADMAP_ERR_INVALID_ARG,
           "extra_index needs n_extra >= 1 and stored single-resolution pointing");
  MM_CHECK(d->n_extra < (1 << 30), MADMAP_ERR_INVALID_ARG, "n_extra too large");
  MM_CHECK(!d->hwp_angle || (d->hwp_tau && d->interval_hwp_group && d->n_hwp_groups >= 1 &&
                             d->n_hwp_groups < (1 << 24) && !d->pix_pol && !d->boresight),
           MADMAP_ERR_INVALID_ARG,
           "hwp_angle needs hwp_tau, interval_hwp_group, n_hwp_groups >= 1 and stored single-resolution pointing");
  if (d->hwp_angle)
    for (int i = 0; i < d->n_intervals; ++i)
      MM_CHECK(d->interval_hwp_group[i] >= -1 && d->interval_hwp_group[i] < d->n_hwp_groups, MADMAP_ERR_INVALID_ARG,
               "interval_hwp_group out of range");
  MM_CHECK(!d->deterministic || (!d->boresight && !d->pix_pol && !d->extra_index && !d->hwp_angle &&
                                  d->n_samples < (1LL << 31) - 1),
           MADMAP_ERR_INVALID_ARG,
           "deterministic plans need stored single-resolution pointing without extended pointing and "
           "n_samples < 2^31");
  MM_CHECK(d->scatter_runs >= -1 && d->scatter_runs <= 1, MADMAP_ERR_INVALID_ARG, "scatter_runs must be -1, 0 or 1");
  MM_CHECK(d->fft_split == 0 || d->fft_split == 1, MADMAP_ERR_INVALID_ARG, "fft_split must be 0 or 1");
  MM_CHECK(!d->allreduce || (!d->boresight && !d->pix_pol && !d->extra_index && !d->hwp_angle),
           MADMAP_ERR_INVALID_ARG, "sharded plans (allreduce set) need stored single-resolution pointing");
  MM_CHECK(d->n_intervals >= 0 && d->interval_offsets != nullptr, MADMAP_ERR_INVALID_ARG, "bad intervals");
  MM_CHECK(d->n_intervals == 0 || d->interval_filter != nullptr, MADMAP_ERR_INVALID_ARG, "interval_filter NULL");
  MM_CHECK(d->n_filters >= 1 && d->n_lags >= 1 && d->filter_lags != nullptr, MADMAP_ERR_INVALID_ARG,
           "need n_filters >= 1, n_lags >= 1 and filter_lags");
  MM_CHECK(d->n_lags <= (1 << 18), MADMAP_ERR_INVALID_ARG, "n_lags too large (max 2^18)");
  const int64_t* off = d->interval_offsets;
  MM_CHECK(off[0] == 0 && off[d->n_intervals] == d->n_samples, MADMAP_ERR_INVALID_ARG,
           "interval_offsets must start at 0 and end at n_samples");
  for (int i = 0; i < d->n_intervals; ++i) {
    MM_CHECK(off[i + 1] >= off[i], MADMAP_ERR_INVALID_ARG, "interval_offsets must be non-decreasing");
    MM_CHECK(d->interval_filter[i] >= 0 && d->interval_filter[i] < d->n_filters, MADMAP_ERR_INVALID_ARG,
             "interval_filter out of range");
  }
  for (long long k = 0; k < (long long)d->n_filters * d->n_lags; ++k)
    MM_CHECK(isfinite(d->filter_lags[k]), MADMAP_ERR_INVALID_ARG, "filter_lags must be finite");
  if (d->fft_len != 0) {
    MM_CHECK(is_pow2(d->fft_len) && d->fft_len >= 256 && d->fft_len <= (1 << 20) &&
                 d->fft_len > 2 * (d->n_lags - 1),
             MADMAP_ERR_INVALID_ARG, "fft_len must be a power of two in [256, 2^20] above 2 (n_lags - 1)");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Plan* p = new Plan();
  p->n_stokes = d->n_stokes;
  p->ns_pad = d->n_stokes == 1 ? 1 : 4;
  p->n_t = d->n_samples;
  p->n_pix = d->n_pix;
  p->n_ivl = d->n_intervals;
  p->n_filters = d->n_filters;
  p->n_lags = d->n_lags;
  p->rcond_excise = d->rcond_excise > 0 ? d->rcond_excise : 1e-6;
  p->rcond_fp64 = d->rcond_fp64 > 0 ? d->rcond_fp64 : 1e-2;
  p->offsets.assign(off, off + d->n_intervals + 1);
  p->ivl_filter.assign(d->interval_filter, d->interval_filter + d->n_intervals);
  p->lags.assign(d->filter_lags, d->filter_lags + (size_t)d->n_filters * d->n_lags);
  p->allreduce = d->allreduce;
  p->allreduce_user = d->allreduce_user;
  madmap_status st = MADMAP_OK;
#define MM_TRY(x)                 \
  do {                            \
    st = (x);                     \
    if (st != MADMAP_OK) {        \
      delete p;                   \
      return st;                  \
    }                             \
  } while (0)
#define MM_TRYC(x) MM_TRY(((x) == cudaSuccess) ? MADMAP_OK : cuda_fail(cudaGetLastError(), #x))
  const long long n = p->n_t;
  const int n_words = (p->n_pix + 31) / 32;
  unsigned* bits = nullptr;
  int* prefix = nullptr;
  int* total = nullptr;
  MM_TRY(dalloc_t(p, &p->dev_flag, 16));
  MM_TRY(dalloc_t(p, &bits, n_words));
  MM_TRY(dalloc_t(p, &prefix, n_words));
  MM_TRY(dalloc_t(p, &total, 2));
  p->otf = otf;
  if (!otf) MM_TRY(dalloc_t(p, &p->pix_obs, std::max(1LL, n)));
  // the second pixelisation of multi-resolution plans
  p->multires = d->pix_pol != nullptr;
  p->n_pix_pol = p->multires ? d->n_pix_pol : 0;
  const int n_words_pol = (p->n_pix_pol + 31) / 32;
  unsigned* bits_pol = nullptr;
  int* prefix_pol = nullptr;
  if (p->multires) {
    MM_TRY(dalloc_t(p, &bits_pol, std::max(1, n_words_pol)));
    MM_TRY(dalloc_t(p, &prefix_pol, std::max(1, n_words_pol)));
    MM_TRY(dalloc_t(p, &p->pix_obs_pol, std::max(1LL, n)));
    MM_TRYC(cudaMemsetAsync(bits_pol, 0, sizeof(unsigned) * std::max(1, n_words_pol), s));
  }
  if (otf) {
    p->n_det = d->n_det;
    p->n_per_det = (int)(n / d->n_det);
    p->bore_step = d->bore_step;
    p->n_bore = d->n_bore;
    p->grid_w = d->grid_width;
    p->grid_h = d->grid_height;
    float4* bore = nullptr;
    MM_TRY(dalloc_t(p, &bore, std::max(1, p->n_bore)));
    if (p->n_bore > 0)
      MM_TRYC(cudaMemcpyAsync(bore, d->boresight, sizeof(float4) * p->n_bore, cudaMemcpyDeviceToDevice, s));
    p->bore = bore;
    MM_TRY(dalloc_t(p, &p->det_pt, p->n_det));
    MM_TRYC(cudaMemcpyAsync(p->det_pt, d->det_pointing, sizeof(float4) * p->n_det, cudaMemcpyHostToDevice, s));
    MM_TRY(dalloc_t(p, &p->g2o, p->n_pix));
  } else if (p->n_stokes == 3) {
    MM_TRY(dalloc_t(p, &p->psi, std::max(1LL, n)));
    MM_TRY(dalloc_t(p, &p->cs64, std::max(1LL, n)));
    MM_TRY(dalloc_t(p, &p->csdf, std::max(1LL, n)));
    MM_TRY(dalloc_t(p, &p->pw, std::max(1LL, n)));
  }
  MM_TRYC(cudaMemsetAsync(p->dev_flag, 0, 16 * sizeof(int), s));
  MM_TRYC(cudaMemsetAsync(bits, 0, sizeof(unsigned) * n_words, s));
  if (otf) {
    if (p->n_bore > 0) k_validate_bore<<<grid_for(p->n_bore), 256, 0, s>>>(p->bore, p->n_bore, p->dev_flag);
    if (n > 0)
      k_mark_bits_otf<<<grid_for(n), 256, 0, s>>>(p->bore, make_step_div(p->bore_step), p->det_pt, p->n_per_det, n,
                                                   p->grid_w, p->grid_h, p->n_stokes == 3, bits);
  } else if (n > 0) {
    k_validate_pix<<<grid_for(n), 256, 0, s>>>(d->pix, n, p->n_pix, p->dev_flag, 1);
    if (p->multires) k_validate_pix<<<grid_for(n), 256, 0, s>>>(d->pix_pol, n, p->n_pix_pol, p->dev_flag, 4);
    if (p->n_stokes == 3) {
      MM_TRYC(cudaMemcpyAsync(p->psi, d->psi, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
      k_validate_psi<<<grid_for(n), 256, 0, s>>>(p->psi, n, p->dev_flag);
    }
    if (!p->allreduce) k_mark_bits<<<grid_for(n), 256, 0, s>>>(d->pix, n, p->n_pix, bits, d->pix_pol);
    if (p->multires) k_mark_bits<<<grid_for(n), 256, 0, s>>>(d->pix_pol, n, p->n_pix_pol, bits_pol, d->pix);
    if (d->extra_index) k_validate_pix<<<grid_for(n), 256, 0, s>>>(d->extra_index, n, d->n_extra, p->dev_flag, 16);
  }
  if (p->allreduce) {
    // sharded plans: a pixel is observed when a sample of any rank hits it
    int* counts = nullptr;
    MM_TRY(dalloc_t(p, &counts, p->n_pix));
    MM_TRYC(cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)p->n_pix, s));
    if (n > 0) k_count_pix<<<grid_for(n), 256, 0, s>>>(d->pix, n, p->n_pix, counts);
    MM_TRY(reduce_across(p, counts, p->n_pix, MADMAP_REDUCE_I32, s));
    k_bits_from_counts<<<grid_for((p->n_pix + 31) / 32), 256, 0, s>>>(counts, p->n_pix, bits);
  }
  k_scan_words<<<1, 1024, 0, s>>>(bits, n_words, prefix, total);
  if (p->multires) k_scan_words<<<1, 1024, 0, s>>>(bits_pol, n_words_pol, prefix_pol, total + 1);
  int hv[3] = {0, 0, 0};
  MM_TRYC(cudaMemcpyAsync(&hv[0], p->dev_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  MM_TRYC(cudaMemcpyAsync(&hv[1], total, sizeof(int) * (p->multires ? 2 : 1), cudaMemcpyDeviceToHost, s));
  MM_TRYC(cudaStreamSynchronize(s));
  MM_TRYC(cudaGetLastError());
  if (hv[0] & 1) {
    delete p;
    set_error("pix holds values outside [-1, n_pix)");
    return MADMAP_ERR_INVALID_ARG;
  }
  if (hv[0] & 2) {
    delete p;
    set_error("psi holds non-finite values");
    return MADMAP_ERR_INVALID_ARG;
  }
  if (hv[0] & 4) {
    delete p;
    set_error("pix_pol holds values outside [-1, n_pix_pol)");
    return MADMAP_ERR_INVALID_ARG;
  }
  if (hv[0] & 8) {
    delete p;
    set_error("boresight holds non-finite values");
    return MADMAP_ERR_INVALID_ARG;
  }
  if (hv[0] & 16) {
    delete p;
    set_error("extra_index holds values outside [-1, n_extra)");
    return MADMAP_ERR_INVALID_ARG;
  }
  p->n_obs_i = hv[1];
  p->n_obs_pol = p->multires ? hv[2] : 0;
  p->n_obs = std::max(p->n_obs_i, p->n_obs_pol);  // map rows (slots for multi-resolution plans)
  if (d->extra_index || d->hwp_angle) {  // extended pointing: extra rows follow the sky rows
    p->ext = true;
    p->n_extra = d->extra_index ? d->n_extra : 0;
    p->n_obs_sky = p->n_obs_i;
    p->n_hwp_groups = d->hwp_angle ? d->n_hwp_groups : 0;
    p->hwp_row0 = p->n_obs_sky + p->n_extra;
    p->n_obs = p->hwp_row0 + 32 * p->n_hwp_groups;
    if (d->extra_index) {
      MM_TRY(dalloc_t(p, &p->ext_row, std::max(1LL, n)));
      if (n > 0) k_ext_rows<<<grid_for(n), 256, 0, s>>>(d->extra_index, n, p->n_obs_sky, p->ext_row);
    }
    if (d->hwp_angle) {
      MM_TRY(dalloc_t(p, &p->hwp_ang, std::max(1LL, n)));
      MM_TRY(dalloc_t(p, &p->hwp_tau, std::max(1LL, n)));
      MM_TRY(dalloc_t(p, &p->hwp_base, std::max(1LL, n)));
      std::vector<int> base(std::max(1, d->n_intervals));
      for (int i = 0; i < d->n_intervals; ++i)
        base[i] = d->interval_hwp_group[i] >= 0 ? p->hwp_row0 + 32 * d->interval_hwp_group[i] : -1;
      int* dbase = nullptr;
      long long* doff = nullptr;
      MM_TRY(dalloc_t(p, &dbase, std::max(1, d->n_intervals)));
      MM_TRY(dalloc_t(p, &doff, d->n_intervals + 1));
      MM_TRYC(cudaMemcpyAsync(dbase, base.data(), sizeof(int) * std::max(1, d->n_intervals), cudaMemcpyHostToDevice, s));
      MM_TRYC(cudaMemcpyAsync(doff, d->interval_offsets, sizeof(long long) * (d->n_intervals + 1),
                              cudaMemcpyHostToDevice, s));
      if (n > 0) {
        MM_TRYC(cudaMemcpyAsync(p->hwp_ang, d->hwp_angle, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
        MM_TRYC(cudaMemcpyAsync(p->hwp_tau, d->hwp_tau, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
        k_hwp_base<<<grid_for(n), 256, 0, s>>>(doff, d->n_intervals, dbase, n, p->hwp_base);
        k_validate_hwp<<<grid_for(n), 256, 0, s>>>(p->hwp_ang, p->hwp_tau, n, p->dev_flag);
      }
      MM_TRYC(cudaStreamSynchronize(s));
      int bad = 0;
      MM_TRYC(cudaMemcpy(&bad, p->dev_flag, sizeof(int), cudaMemcpyDeviceToHost));
      if (bad & 32) {
        delete p;
        set_error("hwp_angle or hwp_tau holds non-finite values");
        return MADMAP_ERR_INVALID_ARG;
      }
    }
  }
  const int n_obs = p->n_obs;
  MM_TRY(dalloc_t(p, &p->obs2glob, std::max(1, p->n_obs_i)));
  MM_TRY(dalloc_t(p, &p->excised, std::max(1, n_obs)));
  MM_TRY(dalloc_t(p, &p->fp64flag, std::max(1, n_obs)));
  MM_TRY(dalloc_t(p, &p->P64, (size_t)std::max(1, n_obs) * (p->n_stokes == 1 ? 1 : 6)));
  MM_TRY(dalloc_t(p, &p->P32, (size_t)std::max(1, n_obs) * (p->n_stokes == 1 ? 1 : 8)));
  k_obs2glob<<<grid_for(p->n_pix), 256, 0, s>>>(bits, prefix, p->n_pix, p->obs2glob);
  if (otf)
    k_g2o<<<grid_for(p->n_pix), 256, 0, s>>>(bits, prefix, p->n_pix, p->g2o);
  else if (n > 0)
    k_pix_obs<<<grid_for(n), 256, 0, s>>>(d->pix, n, p->n_pix, bits, prefix, p->pix_obs, d->pix_pol);
  if (p->multires) {
    MM_TRY(dalloc_t(p, &p->obs2glob_pol, std::max(1, p->n_obs_pol)));
    MM_TRY(dalloc_t(p, &p->excised_pol, std::max(1, n_obs)));
    k_obs2glob<<<grid_for(p->n_pix_pol), 256, 0, s>>>(bits_pol, prefix_pol, p->n_pix_pol, p->obs2glob_pol);
    if (n > 0)
      k_pix_obs<<<grid_for(n), 256, 0, s>>>(d->pix_pol, n, p->n_pix_pol, bits_pol, prefix_pol, p->pix_obs_pol, d->pix);
  }
  MM_TRY(build_preconditioner(p, s));
  if (d->deterministic) {
    p->det = true;
    MM_TRY(build_det_rows(p, s));
  }
  if (p->n_lags == 1) {
    // white noise: runs of at most 2048 samples within each interval
    std::vector<DiagItem> items;
    for (int i = 0; i < p->n_ivl; ++i)
      for (long long t = p->offsets[i]; t < p->offsets[i + 1]; t += 2048)
        items.push_back({t, std::min(p->offsets[i + 1], t + 2048), p->ivl_filter[i], 0});
    p->n_diag_items = (int)items.size();
    MM_CHECK(items.size() < (1ULL << 31), MADMAP_ERR_INVALID_ARG, "too many samples for the white-noise pass");
    MM_TRY(dalloc_t(p, &p->diag_items, std::max<size_t>(1, items.size())));
    if (!items.empty())
      MM_TRYC(cudaMemcpy(p->diag_items, items.data(), sizeof(DiagItem) * items.size(), cudaMemcpyHostToDevice));
    std::vector<double> f0(p->n_filters);
    for (int f = 0; f < p->n_filters; ++f) f0[f] = p->lags[f];
    MM_TRY(dalloc_t(p, &p->f0_64, p->n_filters));
    MM_TRYC(cudaMemcpy(p->f0_64, f0.data(), sizeof(double) * p->n_filters, cudaMemcpyHostToDevice));
    p->diag = true;
  }
  // how often consecutive samples stay in one pixel: the scatter sums such
  // runs within a warp before its atomics when they are common
  if (p->pix_obs && p->n_t > 1) {
    unsigned long long* cnt = nullptr;
    MM_TRY(dalloc_t(p, &cnt, 1));
    MM_TRYC(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
    k_count_repeats<<<grid_for(p->n_t), 256, 0, s>>>(p->pix_obs, p->n_t, cnt);
    unsigned long long h = 0;
    MM_TRYC(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
    MM_TRYC(cudaStreamSynchronize(s));
    p->repeat_frac = (double)h / (double)p->n_t;
  }
  p->runs_fixed = d->scatter_runs != 0;
  p->split_down = d->fft_split;
  p->split_fixed = d->fft_split != 0;
  p->runs = runs_capable(p) && (d->scatter_runs == 1 || (d->scatter_runs == 0 && p->repeat_frac >= kRunsMinFrac))
                ? 1 : 0;
  // FFT geometry and windows: the length and the tiles per launch chunk given
  // in the description, else chosen by the cost model, or by measurement
  {
    const int M0 = d->fft_len ? d->fft_len : choose_fft_len(p->offsets, p->ivl_filter, p->n_filters, p->n_lags);
    if (M0 <= 0) {
      delete p;
      set_error("no FFT length up to 2^20 fits n_lags");
      return MADMAP_ERR_INVALID_ARG;
    }
    if (d->autotune && !p->diag && p->n_t > 0 && p->n_obs > 0)
      MM_TRY(autotune_windows(p, d->fft_len ? d->fft_len : 0, M0, d->tiles_per_chunk, s));
    else
      MM_TRY(setup_windows(p, M0, d->tiles_per_chunk, s));
  }
  if (!p->det && p->n_obs > 0 && p->n_t >= 1024LL * p->n_obs && (long long)p->n_obs * p->ns_pad <= (1LL << 17)) {
    // a small map under more than 1024 samples per row: eight scatter replicas
    p->n_rep = 8;
    const size_t rb = sizeof(double) * (size_t)p->n_rep * p->n_obs * p->ns_pad;
    MM_TRY(dalloc(p, &p->rep, rb));
    MM_TRYC(cudaMemsetAsync(p->rep, 0, rb, s));
  }
  MM_TRYC(cudaStreamSynchronize(s));
  MM_TRYC(cudaGetLastError());
#undef MM_TRY
#undef MM_TRYC
  *out = reinterpret_cast<madmap_plan_t>(p);
  return MADMAP_OK;
}

extern "C" madmap_status madmap_plan_destroy(madmap_plan_t plan) {
  if (!plan) return MADMAP_OK;
  Plan* p = reinterpret_cast<Plan*>(plan);
  cudaDeviceSynchronize();
  delete p;
  return MADMAP_OK;
}

extern "C" madmap_status madmap_plan_get_stats(madmap_plan_t plan, madmap_plan_stats* o) {
  MM_CHECK(plan && o, MADMAP_ERR_INVALID_ARG, "plan_get_stats: NULL argument");
  const Plan* p = reinterpret_cast<const Plan*>(plan);
  o->n_obs = p->n_obs;
  o->n_excised = p->n_excised;
  o->n_fp64_pixels = p->n_fp64;
  o->n_stokes = p->n_stokes;
  o->fft_len = p->M;
  o->n1 = p->N1;
  o->n2 = p->N2;
  o->n_segments = p->n_segments;
  o->n_tiles = p->n_tiles;
  o->tiles_per_chunk = p->tiles_per_chunk;
  o->n_lags = p->n_lags;
  o->n_filters = p->n_filters;
  o->n_samples = p->n_t;
  o->device_bytes = (int64_t)(p->device_bytes + solve_buffer_bytes(p));
  o->n_obs_pol = p->n_obs_pol;
  o->n_excised_pol = p->n_excised_pol;
  o->n_extra = p->n_extra;
  o->n_excised_extra = p->n_excised_extra;
  o->n_hwp_params = 32 * p->n_hwp_groups;
  o->n_excised_hwp = p->n_excised_hwp;
  o->n_map_replicas = p->n_rep;
  o->scatter_runs = p->runs;
  o->repeat_frac = p->repeat_frac;
  o->deterministic = p->det ? 1 : 0;
  o->n_tuned = (int32_t)std::min<size_t>(p->tuned.size(), MADMAP_MAX_TUNED);
  for (int k = 0; k < MADMAP_MAX_TUNED; ++k) {
    const bool has = k < o->n_tuned;
    o->tuned_fft_len[k] = has ? p->tuned[k].M : 0;
    o->tuned_tiles_per_chunk[k] = has ? p->tuned[k].tpc : 0;
    o->tuned_ms[k] = has ? p->tuned[k].ms : 0.f;
    o->tuned_runs[k] = has ? p->tuned[k].runs : 0;
    o->tuned_n2[k] = has ? p->tuned[k].n2 : 0;
  }
  o->sharded = p->allreduce ? 1 : 0;
  return MADMAP_OK;
}

extern "C" madmap_status madmap_plan_observed(madmap_plan_t plan, int32_t* n_obs, int32_t* obs2glob,
                                              uint8_t* excised, void* stream) {
  MM_CHECK(plan, MADMAP_ERR_INVALID_ARG, "plan_observed: NULL plan");
  const Plan* p = reinterpret_cast<const Plan*>(plan);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n_obs) *n_obs = p->n_obs_i;
  if (obs2glob && p->n_obs_i)
    MM_CUDA(cudaMemcpyAsync(obs2glob, p->obs2glob, sizeof(int) * p->n_obs_i, cudaMemcpyDeviceToDevice, s));
  if (excised && p->n_obs_i)
    MM_CUDA(cudaMemcpyAsync(excised, p->excised, p->n_obs_i, cudaMemcpyDeviceToDevice, s));
  return MADMAP_OK;
}

extern "C" madmap_status madmap_plan_observed_pol(madmap_plan_t plan, int32_t* n_obs_pol, int32_t* obs2glob_pol,
                                                  uint8_t* excised_pol, void* stream) {
  MM_CHECK(plan, MADMAP_ERR_INVALID_ARG, "plan_observed_pol: NULL plan");
  const Plan* p = reinterpret_cast<const Plan*>(plan);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n_obs_pol) *n_obs_pol = p->n_obs_pol;
  if (obs2glob_pol && p->n_obs_pol)
    MM_CUDA(cudaMemcpyAsync(obs2glob_pol, p->obs2glob_pol, sizeof(int) * p->n_obs_pol, cudaMemcpyDeviceToDevice, s));
  if (excised_pol && p->n_obs_pol)
    MM_CUDA(cudaMemcpyAsync(excised_pol, p->excised_pol, p->n_obs_pol, cudaMemcpyDeviceToDevice, s));
  return MADMAP_OK;
}

extern "C" madmap_status madmap_plan_expand_pointing(madmap_plan_t plan, int32_t* pix, float* cos2psi,
                                                     float* sin2psi, void* stream) {
  MM_CHECK(plan, MADMAP_ERR_INVALID_ARG, "plan_expand_pointing: NULL plan");
  const Plan* p = reinterpret_cast<const Plan*>(plan);
  MM_CHECK(p->otf, MADMAP_ERR_INVALID_ARG, "plan_expand_pointing: the plan stores its pointing");
  if (p->n_t == 0) return MADMAP_OK;
  const bool pol = p->n_stokes == 3;
  mm::k_expand_all<<<mm::grid_for(p->n_t), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      p->bore, mm::make_step_div(p->bore_step), p->det_pt, p->n_per_det, p->n_t, p->grid_w, p->grid_h, pol, pix,
      pol ? cos2psi : nullptr, pol ? sin2psi : nullptr);
  MM_CUDA(cudaGetLastError());
  return MADMAP_OK;
}

extern "C" madmap_status madmap_plan_set_filters(madmap_plan_t plan, const double* lags, void* stream) {
  MM_CHECK(plan && lags, MADMAP_ERR_INVALID_ARG, "plan_set_filters: NULL argument");
  Plan* p = reinterpret_cast<Plan*>(plan);
  for (long long k = 0; k < (long long)p->n_filters * p->n_lags; ++k)
    MM_CHECK(isfinite(lags[k]), MADMAP_ERR_INVALID_ARG, "filter_lags must be finite");
  std::vector<double> old = p->lags;
  p->lags.assign(lags, lags + (size_t)p->n_filters * p->n_lags);
  madmap_status st = build_spectra(p);
  if (st != MADMAP_OK) {
    p->lags = old;
    build_spectra(p);
    return st;
  }
  if (p->diag) {  // the white-noise pass reads f(0) directly
    MM_CUDA(cudaMemcpy(p->f0_64, p->lags.data(), sizeof(double) * p->n_filters, cudaMemcpyHostToDevice));
  }
  // The block preconditioner weighs samples by f(0) of their filter: rebuild it.
  // Rows of excised pixels are already zero, so those pixels have no hits and
  // classify as excised again; every other pixel keeps its A^T A block.
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return build_preconditioner(p, s);
}
