// PCG solve of H x = b (Section 4, Eq. 10) with MADmap's termination and
// output rule (Section 5): x_0 = 0, stop at max_iter or when the relative
// residual ||r_k|| / ||b|| reaches rel_tol, return the iterate with the lowest
// relative residual seen.  The preconditioner is the per-pixel block inverse
// (A^T W^-1 A)^-1 (Section 5, MADpre).
//
// Each iteration is: q = H p (three operator kernels per tile chunk), then
//   k_cg_alpha      <p,q> -> alpha = <r,z>/<p,q>
//   k_cg_update     x += alpha p, r -= alpha q, z = P r, <r,z>, <r,r> -> beta,
//                   residual, best iterate, termination
//   k_cg_direction  copy x to the best iterate if it improved, p = z + beta p,
//                   q = 0
// Dot products are accumulated in float64 in every precision, per block, and
// the last block to finish (atomic ticket, no waiting) reduces the partials in
// a fixed order, so results are reproducible run to run.  All scalars live on
// the device; the host only reads the state every few iterations.  When the
// solve has finished every kernel returns at once, so chunks of iterations
// can be enqueued (or replayed from a CUDA graph) ahead of the host check.
//
// MIXED precision: float32 operator and vectors inside float64 iterative
// refinement: b and the residual b - H x are float64 (float64 operator), the
// correction solve H e = r runs in float32 with float64 dots and scalars, and
// pixels flagged as poorly conditioned keep float64 preconditioner blocks.
//
// Batched solves (many right-hand sides over one pointing) run every kernel
// with blockIdx.y = right-hand side: vectors, partials and scalars are per
// right-hand side, each stops on its own, and the operator takes a tile set
// whose lanes pair right-hand sides of one window (so they share one FFT and
// one pass over the pointing) and skips tiles whose right-hand sides are done.
#include <math.h>
#include <stdlib.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace mm {

// done: converged, failed or at max_iter.  halt: done, or paused at a
// checkpoint (k >= pause_k); the kernels skip work while halt is set, but the
// search direction of the pausing iteration is still formed.
struct CgState {
  double rz, alpha, beta, bnorm, res, best_res, tol;
  int k, best_k, dir_k, max_iter, done, status, halt, pause_k;
  unsigned counter;
  int pad;
};
static_assert(sizeof(CgState) % sizeof(int) == 0, "per-rhs done flags are strided in ints");
static const int ST_STRIDE = (int)(sizeof(CgState) / sizeof(int));

struct SolveBuffers {
  bool fp64 = false;
  int cap_rhs = 0;
  long long nvec = 0;  // n_obs * ns_pad per right-hand side
  void *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *xb = nullptr;
  double* partials = nullptr;  // [cap_rhs][NB][4]
  CgState* st = nullptr;       // [cap_rhs]
  CgState* host_st = nullptr;  // pinned, 2 slots of cap_rhs
  int* flags = nullptr;        // [cap_rhs] per-rhs skip / inactive flags
  cudaEvent_t ev[2] = {nullptr, nullptr};
  // float64 refinement vectors (allocated with the float64 buffers)
  double *b64 = nullptr, *x64 = nullptr, *r64 = nullptr, *t64 = nullptr, *xbest64 = nullptr;
  df64* xdf = nullptr;  // x64 split into double-float pairs (input of the double-float operator)
  cudaGraphExec_t exec = nullptr;
  int graph_iters = 0, graph_rhs = 0;
  const void* graph_ts = nullptr;
  long long graph_launches = 0;  // kernel nodes per replay
  // device-side loop: a graph whose conditional WHILE node repeats one
  // iteration until every right-hand side is done (or a hard cap is hit)
  cudaGraph_t wgraph = nullptr;
  cudaGraphExec_t wexec = nullptr;
  int w_rhs = 0;
  const void* w_ts = nullptr;
  long long w_body_launches = 0;
  bool w_unsupported = false;
  int* loop = nullptr;  // [0] body executions, [1] cap
  double* hist = nullptr;  // [cap_rhs][HIST_CAP] relative residual after each iteration
  std::vector<void*> allocs;
  size_t bytes = 0;
};

static const int NB = 304;  // blocks of the vector kernels (2 per SM)
static const int HIST_CAP = 4096;  // iterations whose residual is recorded per right-hand side
static const int NT = 256;

static void free_one(SolveBuffers* sb) {
  if (!sb) return;
  if (sb->exec) cudaGraphExecDestroy(sb->exec);
  if (sb->wexec) cudaGraphExecDestroy(sb->wexec);
  if (sb->wgraph) cudaGraphDestroy(sb->wgraph);
  for (int i = 0; i < 2; ++i)
    if (sb->ev[i]) cudaEventDestroy(sb->ev[i]);
  if (sb->host_st) cudaFreeHost(sb->host_st);
  for (void* a : sb->allocs) cudaFree(a);
  delete sb;
}

size_t solve_buffer_bytes(const Plan* p) {
  return (p->sb64 ? p->sb64->bytes : 0) + (p->sb32 ? p->sb32->bytes : 0);
}

void free_solve_buffers(Plan* p) {
  free_one(p->sb64);
  free_one(p->sb32);
  p->sb64 = p->sb32 = nullptr;
}

static madmap_status sb_alloc(Plan* p, SolveBuffers* sb, void** ptr, size_t bytes) {
  madmap_status st = dalloc(p, ptr, bytes);
  if (st != MADMAP_OK) return st;
  // ownership moves to the solve buffers
  p->allocs.pop_back();
  p->device_bytes -= bytes;
  sb->allocs.push_back(*ptr);
  sb->bytes += bytes;
  return MADMAP_OK;
}

// Work buffers for `n_rhs` right-hand sides in one precision (kept with the
// plan and grown when a larger batch arrives).
static madmap_status get_buffers(Plan* p, bool fp64, int n_rhs, SolveBuffers** out) {
  SolveBuffers*& slot = fp64 ? p->sb64 : p->sb32;
  if (slot && slot->cap_rhs >= n_rhs) {
    *out = slot;
    return MADMAP_OK;
  }
  if (slot) {
    cudaDeviceSynchronize();
    free_one(slot);
    slot = nullptr;
  }
  SolveBuffers* sb = new SolveBuffers();
  sb->fp64 = fp64;
  sb->cap_rhs = n_rhs;
  sb->nvec = (long long)std::max(1, p->n_obs) * p->ns_pad;
  const size_t vb = (size_t)sb->nvec * n_rhs * (fp64 ? sizeof(double) : sizeof(float));
  madmap_status st = MADMAP_OK;
  void** vecs[6] = {&sb->x, &sb->r, &sb->z, &sb->p, &sb->q, &sb->xb};
  for (void** v : vecs)
    if ((st = sb_alloc(p, sb, v, vb)) != MADMAP_OK) break;
  if (st == MADMAP_OK) st = sb_alloc(p, sb, (void**)&sb->partials, sizeof(double) * NB * 4 * n_rhs);
  if (st == MADMAP_OK) st = sb_alloc(p, sb, (void**)&sb->st, sizeof(CgState) * n_rhs);
  if (st == MADMAP_OK) st = sb_alloc(p, sb, (void**)&sb->flags, sizeof(int) * n_rhs);
  if (st == MADMAP_OK) st = sb_alloc(p, sb, (void**)&sb->loop, sizeof(int) * 2);
  if (st == MADMAP_OK) st = sb_alloc(p, sb, (void**)&sb->hist, sizeof(double) * HIST_CAP * n_rhs);
  if (st == MADMAP_OK && fp64) {
    double** v64[5] = {&sb->b64, &sb->x64, &sb->r64, &sb->t64, &sb->xbest64};
    for (double** v : v64)
      if ((st = sb_alloc(p, sb, (void**)v, sizeof(double) * sb->nvec * n_rhs)) != MADMAP_OK) break;
    if (st == MADMAP_OK) st = sb_alloc(p, sb, (void**)&sb->xdf, sizeof(df64) * sb->nvec * n_rhs);
  }
  if (st == MADMAP_OK) {
    cudaError_t e = cudaMallocHost(&sb->host_st, 2 * sizeof(CgState) * n_rhs);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sb->ev[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sb->ev[1], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemset(sb->st, 0, sizeof(CgState) * n_rhs);
    if (e != cudaSuccess) st = cuda_fail(e, "solve buffers");
  }
  slot = sb;  // freed with the plan, even when partially built
  if (st != MADMAP_OK) return st;
  *out = sb;
  return MADMAP_OK;
}

// ---------------------------------------------------------------- small vector helpers
template <typename Real, int NS> struct V3 {
  Real a, b, c;
};

template <typename Real, int NS>
__device__ __forceinline__ V3<Real, NS> ldv(const Real* v, int p) {
  V3<Real, NS> o;
  if (NS == 1) {
    o.a = v[p];
    o.b = o.c = 0;
  } else if (sizeof(Real) == 4) {  // one 16-byte load per pixel (the vectors are 16-byte aligned)
    const float4 m = reinterpret_cast<const float4*>(v)[p];
    o.a = (Real)m.x;
    o.b = (Real)m.y;
    o.c = (Real)m.z;
  } else {
    const double2 m0 = reinterpret_cast<const double2*>(v)[2LL * p];
    const double2 m1 = reinterpret_cast<const double2*>(v)[2LL * p + 1];
    o.a = (Real)m0.x;
    o.b = (Real)m0.y;
    o.c = (Real)m1.x;
  }
  return o;
}
template <typename Real, int NS>
__device__ __forceinline__ void stv(Real* v, int p, const V3<Real, NS>& o) {
  if (NS == 1) {
    v[p] = o.a;
  } else if (sizeof(Real) == 4) {
    reinterpret_cast<float4*>(v)[p] = make_float4((float)o.a, (float)o.b, (float)o.c, 0.f);
  } else {
    reinterpret_cast<double2*>(v)[2LL * p] = make_double2((double)o.a, (double)o.b);
    reinterpret_cast<double2*>(v)[2LL * p + 1] = make_double2((double)o.c, 0.0);
  }
}
template <typename Real, int NS>
__device__ __forceinline__ double dotv(const V3<Real, NS>& u, const V3<Real, NS>& v) {
  double s = (double)u.a * (double)v.a;
  if (NS == 3) s += (double)u.b * (double)v.b + (double)u.c * (double)v.c;
  return s;
}

// z = P r with the pixel's block inverse
template <typename Real, int NS>
__device__ __forceinline__ V3<Real, NS> precond(const V3<Real, NS>& r, int p, const double* P64, const float* P32,
                                               const unsigned char* f64) {
  V3<Real, NS> z;
  if (NS == 1) {
    if (sizeof(Real) == 8) z.a = (Real)(P64[p] * (double)r.a);
    else z.a = (Real)(P32[p] * (float)r.a);
    z.b = z.c = 0;
    return z;
  }
  if (sizeof(Real) == 8 || f64[p]) {
    const double* m = P64 + 6LL * p;
    const double a = r.a, b = r.b, c = r.c;
    z.a = (Real)(m[0] * a + m[1] * b + m[2] * c);
    z.b = (Real)(m[1] * a + m[3] * b + m[4] * c);
    z.c = (Real)(m[2] * a + m[4] * b + m[5] * c);
  } else {
    const float4 m0 = reinterpret_cast<const float4*>(P32)[2LL * p];
    const float4 m1 = reinterpret_cast<const float4*>(P32)[2LL * p + 1];
    const float a = r.a, b = r.b, c = r.c;
    z.a = (Real)(m0.x * a + m0.y * b + m0.z * c);
    z.b = (Real)(m0.y * a + m0.w * b + m1.x * c);
    z.c = (Real)(m0.z * a + m1.x * b + m1.y * c);
  }
  return z;
}

// Block sum of up to 2 doubles; returns true in thread 0 of the block that
// finishes last (after every block has published its partials).
template <int K>
__device__ __forceinline__ bool block_reduce_publish(double (&v)[K], double* partials, unsigned* counter) {
  __shared__ double sh[32][K];
  __shared__ bool last;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[wid][k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += sh[w][k];
      partials[blockIdx.x * 4 + k] = s;
    }
    __threadfence();
    const unsigned ticket = atomicAdd(counter, 1u);
    last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  return last;
}

// Sum of all blocks' partials, computed by every thread of the block that
// finished last (block_reduce_publish returned true in all of its threads):
// thread i adds blocks i, i + blockDim.x, ..., then a fixed shuffle tree and
// a fixed pass over the warps combine them, so the result does not depend on
// the order in which blocks finished.  Valid in thread 0.
template <int K>
__device__ __forceinline__ void final_sums(const double* partials, double (&out)[K]) {
  __shared__ double shf[32][K];
  __threadfence();
  double v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] += ((volatile const double*)partials)[b * 4 + k];
#pragma unroll
  for (int k = 0; k < K; ++k)
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) shf[wid][k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      out[k] = 0.0;
      for (int w = 0; w < nw; ++w) out[k] += shf[w][k];
    }
  }
}

// ---------------------------------------------------------------- CG kernels
// All kernels take the right-hand side from blockIdx.y; `nvec` is the length
// of one right-hand side's vectors.
template <typename Real, int NS, typename Bt>
__global__ void __launch_bounds__(NT) k_cg_init(Real* x, Real* r, Real* z, Real* p, Real* q, Real* xb, const Bt* b,
                                                long long nvec, int n_obs, const double* P64, const float* P32,
                                                const unsigned char* f64, CgState* st, double* partials,
                                                double tol, int max_iter, const int* inactive, int pause_k,
                                                double* hist) {
  const long long o = blockIdx.y * nvec;
  x += o; r += o; z += o; p += o; q += o; xb += o; b += o;
  st += blockIdx.y;
  partials += (long long)blockIdx.y * NB * 4;
  double acc[2] = {0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_obs; i += gridDim.x * blockDim.x) {
    V3<Real, NS> rv;
    if (NS == 1) {
      rv.a = (Real)b[i];
      rv.b = rv.c = 0;
    } else {
      rv.a = (Real)b[4LL * i];
      rv.b = (Real)b[4LL * i + 1];
      rv.c = (Real)b[4LL * i + 2];
    }
    const V3<Real, NS> zv = precond<Real, NS>(rv, i, P64, P32, f64);
    const V3<Real, NS> zero = {0, 0, 0};
    stv<Real, NS>(r, i, rv);
    stv<Real, NS>(z, i, zv);
    stv<Real, NS>(p, i, zv);
    stv<Real, NS>(x, i, zero);
    stv<Real, NS>(xb, i, zero);
    stv<Real, NS>(q, i, zero);
    acc[0] += dotv(rv, zv);
    acc[1] += dotv(rv, rv);
  }
  if (block_reduce_publish<2>(acc, partials, &st->counter)) {
    double s[2];
    final_sums<2>(partials, s);
    if (threadIdx.x == 0) {
      st->counter = 0;
      st->rz = s[0];
      st->bnorm = sqrt(s[1]);
      st->res = st->bnorm > 0.0 ? 1.0 : 0.0;
      st->best_res = st->res;
      st->tol = tol;
      st->k = 0;
      st->best_k = 0;
      st->dir_k = 0;
      st->max_iter = max_iter;
      st->status = 0;
      st->alpha = st->beta = 0.0;
      const bool off = inactive && inactive[blockIdx.y];
      st->done = (off || st->bnorm == 0.0 || max_iter <= 0 || st->res <= tol) ? 1 : 0;
      st->pause_k = pause_k;
      st->halt = st->done || pause_k <= 0;
      if (hist) hist[(long long)blockIdx.y * HIST_CAP] = st->res;
    }
  }
}

template <typename Real, int NS>
__global__ void __launch_bounds__(NT) k_cg_alpha(const Real* p, const Real* q, long long nvec, int n_obs,
                                                 CgState* st, double* partials) {
  st += blockIdx.y;
  if (st->halt) return;
  p += blockIdx.y * nvec;
  q += blockIdx.y * nvec;
  partials += (long long)blockIdx.y * NB * 4;
  double acc[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_obs; i += gridDim.x * blockDim.x)
    acc[0] += dotv(ldv<Real, NS>(p, i), ldv<Real, NS>(q, i));
  if (block_reduce_publish<1>(acc, partials, &st->counter)) {
    double s[1];
    final_sums<1>(partials, s);
    if (threadIdx.x == 0) {
      st->counter = 0;
      if (!(s[0] > 0.0) || !isfinite(s[0])) {
        st->status = (int)MADMAP_ERR_NOT_PD;
        st->done = 1;
        st->halt = 1;
      } else {
        st->alpha = st->rz / s[0];
      }
    }
  }
}

template <typename Real, int NS>
__global__ void __launch_bounds__(NT) k_cg_update(Real* x, Real* r, Real* z, const Real* p, const Real* q,
                                                  long long nvec, int n_obs, const double* P64, const float* P32,
                                                  const unsigned char* f64, CgState* st, double* partials,
                                                  double* hist) {
  st += blockIdx.y;
  if (st->halt) return;
  const long long o = blockIdx.y * nvec;
  x += o; r += o; z += o; p += o; q += o;
  partials += (long long)blockIdx.y * NB * 4;
  const Real alpha = (Real)st->alpha;
  double acc[2] = {0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_obs; i += gridDim.x * blockDim.x) {
    V3<Real, NS> xv = ldv<Real, NS>(x, i), rv = ldv<Real, NS>(r, i);
    const V3<Real, NS> pv = ldv<Real, NS>(p, i), qv = ldv<Real, NS>(q, i);
    xv.a += alpha * pv.a;
    rv.a -= alpha * qv.a;
    if (NS == 3) {
      xv.b += alpha * pv.b;
      xv.c += alpha * pv.c;
      rv.b -= alpha * qv.b;
      rv.c -= alpha * qv.c;
    }
    const V3<Real, NS> zv = precond<Real, NS>(rv, i, P64, P32, f64);
    stv<Real, NS>(x, i, xv);
    stv<Real, NS>(r, i, rv);
    stv<Real, NS>(z, i, zv);
    acc[0] += dotv(rv, zv);
    acc[1] += dotv(rv, rv);
  }
  if (block_reduce_publish<2>(acc, partials, &st->counter)) {
    double s[2];
    final_sums<2>(partials, s);
    if (threadIdx.x == 0) {
      st->counter = 0;
      const int k = st->k + 1;
      st->k = k;
      const double res = sqrt(s[1]) / st->bnorm;
      st->res = res;
      if (hist && k < HIST_CAP) hist[(long long)blockIdx.y * HIST_CAP + k] = res;
      if (res < st->best_res) {
        st->best_res = res;
        st->best_k = k;
      }
      if (res <= st->tol || k >= st->max_iter || !isfinite(res)) st->done = 1;
      st->halt = st->done || k >= st->pause_k;
      st->beta = s[0] / st->rz;
      st->rz = s[0];
    }
  }
}

template <typename Real, int NS>
__global__ void __launch_bounds__(NT) k_cg_direction(const Real* x, const Real* z, Real* p, Real* q, Real* xb,
                                                     long long nvec, int n_obs, CgState* st) {
  st += blockIdx.y;
  const int k = st->k;
  if (st->dir_k >= k) return;
  const long long o = blockIdx.y * nvec;
  x += o; z += o; p += o; q += o; xb += o;
  const bool copy = st->best_k == k;
  const bool more = !st->done;
  const Real beta = (Real)st->beta;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_obs; i += gridDim.x * blockDim.x) {
    if (copy) stv<Real, NS>(xb, i, ldv<Real, NS>(x, i));
    if (more) {
      V3<Real, NS> pv = ldv<Real, NS>(p, i);
      const V3<Real, NS> zv = ldv<Real, NS>(z, i);
      pv.a = zv.a + beta * pv.a;
      if (NS == 3) {
        pv.b = zv.b + beta * pv.b;
        pv.c = zv.c + beta * pv.c;
      }
      stv<Real, NS>(p, i, pv);
      const V3<Real, NS> zero = {0, 0, 0};
      stv<Real, NS>(q, i, zero);
    }
  }
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&st->counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    st->counter = 0;
    st->dir_k = k;
  }
}

// Residual replacement: the float32 PCG continues across a refinement step
// (the residual replacement of van der Vorst and Ye, 2000; the "reliable
// updates" of Clark et al., 2010).  The recursive residual is replaced by
// the true residual r64 of the refined float64 iterate, the correction x
// restarts from zero and the search direction is kept.  The new direction is
// made H-conjugate to the last one explicitly, beta = -<z, H p> / <p, H p>
// (the Hestenes-Stiefel form, equal to <r,z> / <r,z>_old when the recursive
// residual is exact), from q = H p of the segment's last iteration, which the
// halted k_cg_direction left in place; k_cg_direction then forms
// p = z + beta p.  The state continues with tolerance (relative to the first
// segment's ||b||) max(inner_tol * its new relative residual, floor_tol) and
// `budget` more iterations.
template <typename Real, int NS>
__global__ void __launch_bounds__(NT) k_cg_replace(Real* x, Real* r, Real* z, Real* xb, const Real* p, const Real* q,
                                                   const double* r64, long long nvec, int n_obs, const double* P64,
                                                   const float* P32, const unsigned char* f64, CgState* st,
                                                   double* partials, double inner_tol, double floor_tol, int budget,
                                                   const int* inactive, double* hist) {
  if (inactive && inactive[blockIdx.y]) return;
  st += blockIdx.y;
  const long long o = blockIdx.y * nvec;
  x += o; r += o; z += o; xb += o; p += o; q += o; r64 += o;
  partials += (long long)blockIdx.y * NB * 4;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_obs; i += gridDim.x * blockDim.x) {
    const V3<double, NS> t = ldv<double, NS>(r64, i);
    V3<Real, NS> rv;
    rv.a = (Real)t.a;
    rv.b = (Real)t.b;
    rv.c = (Real)t.c;
    const V3<Real, NS> zv = precond<Real, NS>(rv, i, P64, P32, f64);
    const V3<Real, NS> pv = ldv<Real, NS>(p, i), qv = ldv<Real, NS>(q, i);
    const V3<Real, NS> zero = {0, 0, 0};
    stv<Real, NS>(r, i, rv);
    stv<Real, NS>(z, i, zv);
    stv<Real, NS>(x, i, zero);
    stv<Real, NS>(xb, i, zero);
    acc[0] += dotv(rv, zv);
    acc[1] += dotv(rv, rv);
    acc[2] += dotv(zv, qv);
    acc[3] += dotv(pv, qv);
  }
  if (block_reduce_publish<4>(acc, partials, &st->counter)) {
    double s[4];
    final_sums<4>(partials, s);
    if (threadIdx.x == 0) {
      st->counter = 0;
      const int k = st->k;
      const double res = sqrt(s[1]) / st->bnorm;
      st->beta = (s[3] > 0.0 && isfinite(s[2] / s[3])) ? -s[2] / s[3] : 0.0;
      st->rz = s[0];
      st->res = res;
      st->best_res = res;
      st->best_k = k;
      st->dir_k = k - 1;
      const double tol = fmax(inner_tol * res, floor_tol);
      st->tol = tol;
      st->max_iter = k + (budget > 0 ? budget : 0);
      st->status = 0;
      st->done = (res <= tol || budget <= 0 || !(s[0] > 0.0)) ? 1 : 0;
      st->halt = st->done;
      if (hist && k < HIST_CAP) hist[(long long)blockIdx.y * HIST_CAP + k] = res;
    }
  }
}

// ---------------------------------------------------------------- layout and refinement kernels
// user [n][ns] (U) -> padded working layout [n][ns_pad] (Real)
template <typename U, typename Real>
__global__ void k_pack(const U* in, Real* out, int n_obs, int ns, int ns_pad) {
  const long long n = (long long)n_obs * ns_pad;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i % ns_pad);
    const long long pp = i / ns_pad;
    out[i] = s < ns ? (Real)in[pp * ns + s] : (Real)0;
  }
}
template <typename Real, typename U>
__global__ void k_unpack(const Real* in, U* out, int n_obs, int ns, int ns_pad) {
  const long long n = (long long)n_obs * ns;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i % ns);
    const long long pp = i / ns;
    out[i] = (U)in[pp * ns_pad + s];
  }
}

// x64 += e (float32 correction) for active right-hand sides, t64 = 0
__global__ void k_refine_add(double* x64, const float* e, double* t64, long long nvec, const int* inactive) {
  if (inactive && inactive[blockIdx.y]) return;
  const long long o = blockIdx.y * nvec;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nvec; i += (long long)gridDim.x * blockDim.x) {
    x64[o + i] += (double)e[o + i];
    t64[o + i] = 0.0;
  }
}

// y = x as double-float pairs
__global__ void k_split(const double* x, df64* y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = df64(x[i]);
}

// Arithmetic of the right-hand side and the refinement residuals.
static int refine_prec(const madmap_solve_opts& o) {
  return (o.precision == MADMAP_MIXED && o.refine_precision == MADMAP_DF64) ? OPP_DF64 : OPP_F64;
}

// Mixed solves of single-resolution stored pointing compute each refinement
// residual b - H x as A^T N^-1 (d - A x) in one full-precision operator
// application (the difference taken per sample before the noise weighting),
// so the right-hand side itself only starts the first float32 inner solve and
// is formed in float32.
static bool fused_residual(const Plan* p, const madmap_solve_opts& o) {
  return o.precision == MADMAP_MIXED && !p->otf && !p->ext && !p->multires;
}

// y = (double) x
__global__ void k_widen(const float* x, double* y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

// r64 = b64 - t64 and ||r64|| -> st[rhs].res (by the last block of the rhs)
__global__ void __launch_bounds__(NT) k_residual(const double* b64, const double* t64, double* r64, long long nvec,
                                                 CgState* st, double* partials, const int* inactive) {
  if (inactive && inactive[blockIdx.y]) return;
  const long long o = blockIdx.y * nvec;
  st += blockIdx.y;
  partials += (long long)blockIdx.y * NB * 4;
  double acc[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nvec; i += (long long)gridDim.x * blockDim.x) {
    const double v = b64[o + i] - t64[o + i];
    r64[o + i] = v;
    acc[0] += v * v;
  }
  if (block_reduce_publish<1>(acc, partials, &st->counter)) {
    double s[1];
    final_sums<1>(partials, s);
    if (threadIdx.x == 0) {
      st->counter = 0;
      st->res = sqrt(s[0]);
    }
  }
}

// xbest64 = x64 for right-hand sides flagged in `take`
__global__ void k_take_best(const double* x64, double* xbest64, long long nvec, const int* take) {
  if (!take[blockIdx.y]) return;
  const long long o = blockIdx.y * nvec;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nvec; i += (long long)gridDim.x * blockDim.x)
    xbest64[o + i] = x64[o + i];
}

static int grid_vec(long long n) {
  long long g = (n + NT - 1) / NT;
  return (int)std::max(1LL, std::min<long long>(g, NB));
}

// ---------------------------------------------------------------- PCG driver
struct Batch {
  int n_rhs = 1;
  const TileSet* ts = nullptr;  // NULL: single right-hand side over the plan's own tiles
};

template <typename Real, int NS>
static void enqueue_iteration(Plan* p, SolveBuffers* sb, const Batch& B, cudaStream_t s, madmap_status* st) {
  Real* x = (Real*)sb->x;
  Real* r = (Real*)sb->r;
  Real* z = (Real*)sb->z;
  Real* pp = (Real*)sb->p;
  Real* q = (Real*)sb->q;
  Real* xb = (Real*)sb->xb;
  const int n = p->n_obs;
  const long long nv = sb->nvec;
  const dim3 g(grid_vec(n), B.n_rhs);
  if (B.ts)
    *st = op_launch_set(p, sizeof(Real) == 8, IN_MAP, OUT_MAP, pp, q, nv, nv, &sb->st->halt, ST_STRIDE, B.ts, s);
  else
    *st = op_launch(p, sizeof(Real) == 8, IN_MAP, OUT_MAP, pp, q, 0, 0, 1, &sb->st->halt, s);
  // sharded plans: q = sum over the ranks of their shares of H p
  if (*st == MADMAP_OK)
    *st = reduce_across(p, q, nv * B.n_rhs, sizeof(Real) == 8 ? MADMAP_REDUCE_F64 : MADMAP_REDUCE_F32, s);
  count_launches(3);
  k_cg_alpha<Real, NS><<<g, NT, 0, s>>>(pp, q, nv, n, sb->st, sb->partials);
  k_cg_update<Real, NS><<<g, NT, 0, s>>>(x, r, z, pp, q, nv, n, p->P64, p->P32, p->fp64flag, sb->st, sb->partials,
                                         sb->hist);
  k_cg_direction<Real, NS><<<g, NT, 0, s>>>(x, z, pp, q, xb, nv, n, sb->st);
}

template <typename Real, int NS>
static madmap_status enqueue_chunk(Plan* p, SolveBuffers* sb, const Batch& B, int iters, bool use_graph,
                                   cudaStream_t s) {
  madmap_status st = MADMAP_OK;
  if (!use_graph) {
    for (int i = 0; i < iters && st == MADMAP_OK; ++i) enqueue_iteration<Real, NS>(p, sb, B, s, &st);
    return st;
  }
  if (!sb->exec || sb->graph_iters != iters || sb->graph_rhs != B.n_rhs || sb->graph_ts != (const void*)B.ts) {
    // kernel attributes are set before capture begins
    st = op_launch(p, sizeof(Real) == 8, IN_MAP, OUT_MAP, nullptr, nullptr, 0, 0, 0, nullptr, s);
    if (st != MADMAP_OK) return st;
    if (sb->exec) {
      cudaGraphExecDestroy(sb->exec);
      sb->exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    const int64_t before = madmap_kernel_launch_count();
    MM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    for (int i = 0; i < iters && st == MADMAP_OK; ++i) enqueue_iteration<Real, NS>(p, sb, B, s, &st);
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    // captured kernels did not run: count them once per replay instead
    sb->graph_launches = madmap_kernel_launch_count() - before;
    count_launches(-sb->graph_launches);
    if (st != MADMAP_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    MM_CUDA(e);
    e = cudaGraphInstantiate(&sb->exec, graph, 0);
    cudaGraphDestroy(graph);
    MM_CUDA(e);
    sb->graph_iters = iters;
    sb->graph_rhs = B.n_rhs;
    sb->graph_ts = B.ts;
  }
  MM_CUDA(cudaGraphLaunch(sb->exec, s));
  count_launches(sb->graph_launches);
  return MADMAP_OK;
}

// Condition of the device-side loop: continue while some right-hand side is
// not done, and never beyond the cap (loop[1]) iterations.
__global__ void k_loop_cond(const CgState* st, int n_rhs, int* loop, cudaGraphConditionalHandle h) {
  int live = 0;
  for (int r = threadIdx.x; r < n_rhs; r += 32) live |= !st[r].halt;
  live = __any_sync(0xffffffffu, live);
  if (threadIdx.x == 0) {
    const int it = loop[0] + 1;
    loop[0] = it;
    cudaGraphSetConditional(h, (live && it < loop[1]) ? 1u : 0u);
  }
}

template <typename Real, int NS>
static madmap_status build_while_graph(Plan* p, SolveBuffers* sb, const Batch& B, cudaStream_t s) {
  if (sb->wexec && sb->w_rhs == B.n_rhs && sb->w_ts == (const void*)B.ts) return MADMAP_OK;
  if (sb->wexec) {
    cudaGraphExecDestroy(sb->wexec);
    sb->wexec = nullptr;
  }
  if (sb->wgraph) {
    cudaGraphDestroy(sb->wgraph);
    sb->wgraph = nullptr;
  }
  madmap_status st = op_launch(p, sizeof(Real) == 8, IN_MAP, OUT_MAP, nullptr, nullptr, 0, 0, 0, nullptr, s);
  if (st != MADMAP_OK) return st;
  cudaGraph_t g = nullptr;
  MM_CUDA(cudaGraphCreate(&g, 0));
  sb->wgraph = g;
  cudaGraphConditionalHandle h;
  MM_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault));
  // zeroed storage: the parameter union has no default constructor
  alignas(cudaGraphNodeParams) unsigned char np_raw[sizeof(cudaGraphNodeParams)] = {};
  cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(np_raw);
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  MM_CUDA(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  const int64_t before = madmap_kernel_launch_count();
  MM_CUDA(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  enqueue_iteration<Real, NS>(p, sb, B, s, &st);
  k_loop_cond<<<1, 32, 0, s>>>(sb->st, B.n_rhs, sb->loop, h);
  cudaGraph_t captured = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s, &captured);
  sb->w_body_launches = madmap_kernel_launch_count() - before + 1;
  count_launches(-(sb->w_body_launches - 1));
  if (st != MADMAP_OK) return st;
  MM_CUDA(e);
  MM_CUDA(cudaGraphInstantiate(&sb->wexec, g, 0));
  sb->w_rhs = B.n_rhs;
  sb->w_ts = B.ts;
  return MADMAP_OK;
}

struct PcgResult {
  int iters = 0, best_iter = 0, status = 0;
  double best_res = 0.0, final_res = 0.0;
};

// Runs PCG on H e = b for every right-hand side of the batch, in the buffers'
// precision.  b: Bt vectors in the padded working layout, nvec apart.
// inactive (device, may be NULL): right-hand sides to leave untouched.
// Results: best iterates in sb->xb, summaries in out[rhs].
// pause_k: iteration at which to halt for a checkpoint (INT_MAX: never).
// init = false continues from the state already in the buffers (a resumed or
// paused solve) instead of starting from x = 0.
template <typename Real, int NS, typename Bt>
static madmap_status run_pcg(Plan* p, SolveBuffers* sb, const Batch& B, const Bt* b, const int* inactive, double tol,
                             int max_iter, int per_sync, int graph_mode, cudaStream_t s, std::vector<PcgResult>& out,
                             int pause_k = INT_MAX, bool init = true) {
  const int n = p->n_obs, R = B.n_rhs;
  if (p->allreduce) graph_mode = 0;  // the cross-rank sums run on the host between launches
  if (init) {
    count_launches(1);
    k_cg_init<Real, NS, Bt><<<dim3(grid_vec(n), R), NT, 0, s>>>(
        (Real*)sb->x, (Real*)sb->r, (Real*)sb->z, (Real*)sb->p, (Real*)sb->q, (Real*)sb->xb, b, sb->nvec, n, p->P64,
        p->P32, p->fp64flag, sb->st, sb->partials, tol, max_iter, inactive, pause_k, sb->hist);
    MM_CUDA(cudaGetLastError());
  }
  if (graph_mode == 2 && !sb->w_unsupported) {
    // one graph launch runs every iteration on the device
    if (build_while_graph<Real, NS>(p, sb, B, s) != MADMAP_OK) {
      // conditional graph nodes unavailable here: fall back to host-checked chunks
      sb->w_unsupported = true;
      cudaGetLastError();
      cudaStreamCaptureStatus cs;
      if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        cudaGraph_t junk = nullptr;
        cudaStreamEndCapture(s, &junk);
        if (junk) cudaGraphDestroy(junk);
      }
    } else {
      const int ctl[2] = {0, max_iter + 2};
      MM_CUDA(cudaMemcpyAsync(sb->loop, ctl, sizeof(ctl), cudaMemcpyHostToDevice, s));
      MM_CUDA(cudaGraphLaunch(sb->wexec, s));
      int ran[2] = {0, 0};
      MM_CUDA(cudaMemcpyAsync(ran, sb->loop, sizeof(ran), cudaMemcpyDeviceToHost, s));
      std::vector<CgState> h(R);
      MM_CUDA(cudaMemcpyAsync(h.data(), sb->st, sizeof(CgState) * R, cudaMemcpyDeviceToHost, s));
      MM_CUDA(cudaStreamSynchronize(s));
      count_launches((long long)ran[0] * sb->w_body_launches);
      out.assign(R, PcgResult());
      for (int k = 0; k < R; ++k) {
        out[k].iters = h[k].k;
        out[k].best_iter = h[k].best_k;
        out[k].best_res = h[k].best_res;
        out[k].final_res = h[k].res;
        out[k].status = h[k].status;
      }
      return MADMAP_OK;
    }
  }
  const bool use_graph = graph_mode != 0;
  int launched = 0, slot = 0;
  bool pending = false;
  const int G = std::max(1, per_sync);
  auto all_done = [&](int sl) {
    for (int k = 0; k < R; ++k)
      if (!sb->host_st[sl * sb->cap_rhs + k].halt) return false;
    return true;
  };
  // one chunk in flight ahead of the host check
  while (true) {
    if (launched < max_iter) {
      madmap_status st = enqueue_chunk<Real, NS>(p, sb, B, G, use_graph, s);
      if (st != MADMAP_OK) return st;
      launched += G;
    }
    MM_CUDA(cudaMemcpyAsync(&sb->host_st[slot * sb->cap_rhs], sb->st, sizeof(CgState) * R, cudaMemcpyDeviceToHost, s));
    MM_CUDA(cudaEventRecord(sb->ev[slot], s));
    if (pending) {
      const int prev = slot ^ 1;
      MM_CUDA(cudaEventSynchronize(sb->ev[prev]));
      if (all_done(prev)) break;
    }
    if (launched >= max_iter && pending) {
      MM_CUDA(cudaEventSynchronize(sb->ev[slot]));
      break;
    }
    pending = true;
    slot ^= 1;
  }
  MM_CUDA(cudaStreamSynchronize(s));
  std::vector<CgState> h(R);
  MM_CUDA(cudaMemcpy(h.data(), sb->st, sizeof(CgState) * R, cudaMemcpyDeviceToHost));
  out.assign(R, PcgResult());
  for (int k = 0; k < R; ++k) {
    out[k].iters = h[k].k;
    out[k].best_iter = h[k].best_k;
    out[k].best_res = h[k].best_res;
    out[k].final_res = h[k].res;
    out[k].status = h[k].status;
  }
  return MADMAP_OK;
}

// PCG (FP64) or refined mixed-precision PCG (MIXED) on H x = b for every
// right-hand side of the batch, b already in sb64->b64.  On return *x_pad
// points at the best iterates (padded layout, nvec apart) and I holds the
// per-rhs summaries (fp64_applies counts the right-hand side's own as 1).
// Copies the float64 solver state (single right-hand side) to a checkpoint:
// the padded device vectors are unpacked through b64, which the float64 PCG
// no longer needs once started.
template <int NS>
static madmap_status write_checkpoint(Plan* p, SolveBuffers* sb, const CgState& h, madmap_checkpoint* c,
                                      cudaStream_t s) {
  const int n = p->n_obs, ns = p->n_stokes, np = p->ns_pad;
  const long long user = (long long)n * ns;
  const double* src[5] = {(const double*)sb->x, (const double*)sb->r, (const double*)sb->z, (const double*)sb->p,
                          (const double*)sb->xb};
  double* dst[5] = {c->x, c->r, c->z, c->p, c->x_best};
  for (int k = 0; k < 5; ++k) {
    count_launches(1);
    k_unpack<double, double><<<grid_vec(user), NT, 0, s>>>(src[k], sb->b64, n, ns, np);
    MM_CUDA(cudaMemcpyAsync(dst[k], sb->b64, sizeof(double) * user, cudaMemcpyDeviceToHost, s));
  }
  MM_CUDA(cudaStreamSynchronize(s));
  c->n_obs = n;
  c->n_stokes = ns;
  c->iters = h.k;
  c->best_iter = h.best_k;
  c->rz = h.rz;
  c->bnorm = h.bnorm;
  c->rel_res = h.res;
  c->best_rel_res = h.best_res;
  return MADMAP_OK;
}

// Float64 PCG, in segments of opts.checkpoint_every iterations when
// checkpoints are requested: at each pause the state is written to
// opts.checkpoint and opts.on_checkpoint may stop the solve (*stopped = 1).
// init = false continues from the state in the buffers (a resume).
template <int NS>
static madmap_status pcg64(Plan* p, SolveBuffers* sb, const Batch& B, const madmap_solve_opts& o, cudaStream_t s,
                           std::vector<PcgResult>& R, bool init, int first_pause, int* stopped) {
  const int every = (o.checkpoint_every > 0 && B.n_rhs == 1) ? o.checkpoint_every : 0;
  int pause = every ? first_pause : INT_MAX;
  *stopped = 0;
  while (true) {
    madmap_status st = run_pcg<double, NS, double>(p, sb, B, sb->b64, nullptr, o.rel_tol, o.max_iter,
                                                   o.iters_per_sync, o.use_graph, s, R, pause, init);
    if (st != MADMAP_OK) return st;
    init = false;
    if (!every) return MADMAP_OK;
    CgState h;
    MM_CUDA(cudaMemcpy(&h, sb->st, sizeof(CgState), cudaMemcpyDeviceToHost));
    if (h.done) return MADMAP_OK;
    st = write_checkpoint<NS>(p, sb, h, o.checkpoint, s);
    if (st != MADMAP_OK) return st;
    if (o.on_checkpoint && o.on_checkpoint(o.checkpoint, o.checkpoint_user) != 0) {
      *stopped = 1;
      return MADMAP_OK;
    }
    pause = h.k + every;
    const int ctl[2] = {0, pause};  // halt, pause_k
    MM_CUDA(cudaMemcpyAsync(&sb->st->halt, ctl, sizeof(ctl), cudaMemcpyHostToDevice, s));
  }
}

// Entries [from, to] of right-hand side k's device residual history, appended
// to `out` multiplied by `scale` (entries past the recorded capacity are not kept).
static madmap_status append_hist(SolveBuffers* sb, int k, int from, int to, double scale, std::vector<double>& out,
                                 cudaStream_t s) {
  to = std::min(to, HIST_CAP - 1);
  if (to < from) return MADMAP_OK;
  std::vector<double> h((size_t)(to - from + 1));
  MM_CUDA(cudaMemcpyAsync(h.data(), sb->hist + (long long)k * HIST_CAP + from, sizeof(double) * h.size(),
                          cudaMemcpyDeviceToHost, s));
  MM_CUDA(cudaStreamSynchronize(s));
  for (double v : h) out.push_back(v * scale);
  return MADMAP_OK;
}

// The residual histories into the caller's buffer (opts.residual_history).
static void write_hist(const madmap_solve_opts& o, const std::vector<std::vector<double>>& H,
                       std::vector<madmap_solve_info>& I) {
  for (size_t k = 0; k < H.size(); ++k) {
    int len = 0;
    if (o.residual_history && o.history_capacity > 0) {
      len = (int)std::min<size_t>(H[k].size(), (size_t)o.history_capacity);
      if (len > 0) memcpy(o.residual_history + (long long)k * o.history_capacity, H[k].data(), sizeof(double) * len);
    }
    I[k].history_len = len;
  }
}

static double ms_since(std::chrono::steady_clock::time_point t) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t).count();
}

// d (device float [n_rhs][n_t], or NULL when b does not come from data, as in
// the adjoint solve): mixed solves then compute their refinement residuals
// from d (fused_residual).
template <int NS>
static madmap_status solve_core(Plan* p, const Batch& B, SolveBuffers* sb64, const madmap_solve_opts& o,
                                std::vector<madmap_solve_info>& I, cudaStream_t s, const double** x_pad,
                                const float* d = nullptr) {
  const int n_rhs = B.n_rhs;
  const long long nv = sb64->nvec;
  const dim3 gv(grid_vec(nv), n_rhs);
  const int graph = o.use_graph;
  madmap_status st = MADMAP_OK;
  std::vector<PcgResult> R;
  const bool want_hist = o.residual_history && o.history_capacity > 0;
  std::vector<std::vector<double>> Hh(n_rhs);
  if (o.precision == MADMAP_FP64) {
    int stopped = 0;
    const auto t_pcg = std::chrono::steady_clock::now();
    st = pcg64<NS>(p, sb64, B, o, s, R, true, o.checkpoint_every, &stopped);
    if (st != MADMAP_OK) return st;
    const double pcg_ms = ms_since(t_pcg);
    for (int k = 0; k < n_rhs && want_hist; ++k)
      if ((st = append_hist(sb64, k, 0, R[k].iters, 1.0, Hh[k], s)) != MADMAP_OK) return st;
    write_hist(o, Hh, I);
    for (int k = 0; k < n_rhs; ++k) {
      I[k].t_pcg_ms = pcg_ms;
      I[k].iters = R[k].iters;
      I[k].outer_iters = 1;
      I[k].best_iter = R[k].best_iter;
      I[k].fp64_applies += R[k].iters;
      I[k].final_rel_res = R[k].final_res;
      I[k].best_rel_res = R[k].best_res;
      I[k].status = R[k].status != 0 ? R[k].status : (R[k].best_res <= o.rel_tol ? MADMAP_OK : MADMAP_WARN_MAXITER);
      if (stopped && I[k].status == MADMAP_WARN_MAXITER) I[k].status = MADMAP_STOPPED;
    }
    *x_pad = (const double*)sb64->xb;
    return MADMAP_OK;
  }
  SolveBuffers* sb32 = nullptr;
  st = get_buffers(p, false, n_rhs, &sb32);
  if (st != MADMAP_OK) return st;
  // r64 = b64 and ||b|| per right-hand side
  MM_CUDA(cudaMemsetAsync(sb64->t64, 0, sizeof(double) * nv * n_rhs, s));
  count_launches(1);
  k_residual<<<gv, NT, 0, s>>>(sb64->b64, sb64->t64, sb64->r64, nv, sb64->st, sb64->partials, nullptr);
  std::vector<CgState> h(n_rhs);
  MM_CUDA(cudaMemcpyAsync(h.data(), sb64->st, sizeof(CgState) * n_rhs, cudaMemcpyDeviceToHost, s));
  MM_CUDA(cudaStreamSynchronize(s));
  std::vector<double> bnorm(n_rhs), best(n_rhs), res(n_rhs);
  std::vector<int> total(n_rhs, 0), best_iter(n_rhs, 0), inner_status(n_rhs, 0), inactive(n_rhs), take(n_rhs);
  int n_active = 0;
  for (int k = 0; k < n_rhs; ++k) {
    bnorm[k] = h[k].res;
    best[k] = res[k] = bnorm[k] > 0 ? 1.0 : 0.0;
    inactive[k] = !(bnorm[k] > 0 && res[k] > o.rel_tol && o.max_iter > 0);
    n_active += !inactive[k];
    if (want_hist) Hh[k].push_back(res[k]);
  }
  double pcg_ms = 0.0, refine_ms = 0.0;
  MM_CUDA(cudaMemsetAsync(sb64->x64, 0, sizeof(double) * nv * n_rhs, s));
  MM_CUDA(cudaMemsetAsync(sb64->xbest64, 0, sizeof(double) * nv * n_rhs, s));
  // continued inner PCG (residual replacement, k_cg_replace): iterations so far
  // of each right-hand side's one float32 PCG, and no step below rel_tol / 2
  const bool cont = !o.inner_restart;
  const double floor_tol = cont ? 0.5 * o.rel_tol : 0.0;
  std::vector<int> kdone(n_rhs, 0), seg(n_rhs, 0);
  int outer = 0;
  while (n_active > 0 && outer < o.max_outer) {
    int budget = 0;
    for (int k = 0; k < n_rhs; ++k)
      if (!inactive[k]) budget = std::max(budget, o.max_iter - total[k]);
    MM_CUDA(cudaMemcpyAsync(sb64->flags, inactive.data(), sizeof(int) * n_rhs, cudaMemcpyHostToDevice, s));
    const auto t_pcg = std::chrono::steady_clock::now();
    if (cont && outer > 0) {
      const int n = p->n_obs;
      const dim3 g(grid_vec(n), n_rhs);
      count_launches(2);
      k_cg_replace<float, NS><<<g, NT, 0, s>>>((float*)sb32->x, (float*)sb32->r, (float*)sb32->z, (float*)sb32->xb,
                                               (const float*)sb32->p, (const float*)sb32->q, sb64->r64, sb32->nvec,
                                               n, p->P64, p->P32, p->fp64flag, sb32->st, sb32->partials,
                                               o.inner_rel_tol, floor_tol, budget, sb64->flags, sb32->hist);
      k_cg_direction<float, NS><<<g, NT, 0, s>>>((const float*)sb32->x, (const float*)sb32->z, (float*)sb32->p,
                                                 (float*)sb32->q, (float*)sb32->xb, sb32->nvec, n, sb32->st);
      MM_CUDA(cudaGetLastError());
      st = run_pcg<float, NS, double>(p, sb32, B, sb64->r64, sb64->flags, 0.0, budget, o.iters_per_sync, graph, s,
                                      R, INT_MAX, false);
    } else {
      st = run_pcg<float, NS, double>(p, sb32, B, sb64->r64, sb64->flags, std::max(o.inner_rel_tol, floor_tol),
                                      budget, o.iters_per_sync, graph, s, R);
    }
    if (st != MADMAP_OK) return st;
    pcg_ms += ms_since(t_pcg);
    const auto t_ref = std::chrono::steady_clock::now();
    for (int k = 0; k < n_rhs; ++k) {
      if (inactive[k]) continue;
      seg[k] = R[k].iters - (cont ? kdone[k] : 0);   // this step's inner iterations
      if (want_hist) {
        st = cont ? append_hist(sb32, k, kdone[k] + 1, R[k].iters, 1.0, Hh[k], s)
                  : append_hist(sb32, k, 1, R[k].iters, res[k], Hh[k], s);
        if (st != MADMAP_OK) return st;
      }
      if (cont) kdone[k] = R[k].iters;
    }
    const int step = outer++;
    count_launches(2);
    // the continued PCG's current iterate carries its residual and direction;
    // a restarted step's best iterate
    k_refine_add<<<gv, NT, 0, s>>>(sb64->x64, (const float*)(cont ? sb32->x : sb32->xb), sb64->t64, nv,
                                   sb64->flags);
    // a continued step that started from a replaced residual and reached
    // rel_tol stops on its recursive residual (no full-precision residual)
    std::vector<int> acc(n_rhs, 0);
    int n_acc = 0;
    if (cont && !o.final_residual && step >= 1) {
      std::vector<int> skip(inactive);
      for (int k = 0; k < n_rhs; ++k)
        if (!inactive[k] && R[k].status == 0 && seg[k] > 0 && R[k].final_res <= o.rel_tol) {
          acc[k] = skip[k] = 1;
          ++n_acc;
        }
      if (n_acc) MM_CUDA(cudaMemcpyAsync(sb64->flags, skip.data(), sizeof(int) * n_rhs, cudaMemcpyHostToDevice, s));
    }
    const int rp = refine_prec(o);
    const void* xin = sb64->x64;
    const bool need_res = n_acc < n_active;
    if (need_res && rp == OPP_DF64) {
      count_launches(1);
      k_split<<<grid_vec(nv * n_rhs), NT, 0, s>>>(sb64->x64, sb64->xdf, nv * n_rhs);
      xin = sb64->xdf;
    }
    if (!need_res) {
      // every active right-hand side stopped on its recursive residual
    } else if (d && fused_residual(p, o)) {
      // r = A^T N^-1 (d - A x) in one pass; t64 (zero since k_refine_add) stands in for H x
      MM_CUDA(cudaMemsetAsync(sb64->r64, 0, sizeof(double) * nv * n_rhs, s));
      p->resid_d = d;
      p->resid_stride = p->n_t;
      if (B.ts)
        st = op_launch_set(p, rp, IN_RESID, OUT_MAP, xin, sb64->r64, nv, nv, sb64->flags, 1, B.ts, s);
      else
        st = op_launch(p, rp, IN_RESID, OUT_MAP, xin, sb64->r64, 0, 0, 1, nullptr, s);
      p->resid_d = nullptr;
      p->resid_stride = 0;
      if (st == MADMAP_OK) st = reduce_across(p, sb64->r64, nv * n_rhs, MADMAP_REDUCE_F64, s);
      if (st != MADMAP_OK) return st;
      k_residual<<<gv, NT, 0, s>>>(sb64->r64, sb64->t64, sb64->r64, nv, sb64->st, sb64->partials, sb64->flags);
    } else {
      if (B.ts)
        st = op_launch_set(p, rp, IN_MAP, OUT_MAP, xin, sb64->t64, nv, nv, sb64->flags, 1, B.ts, s);
      else
        st = op_launch(p, rp, IN_MAP, OUT_MAP, xin, sb64->t64, 0, 0, 1, nullptr, s);
      if (st == MADMAP_OK) st = reduce_across(p, sb64->t64, nv * n_rhs, MADMAP_REDUCE_F64, s);
      if (st != MADMAP_OK) return st;
      k_residual<<<gv, NT, 0, s>>>(sb64->b64, sb64->t64, sb64->r64, nv, sb64->st, sb64->partials, sb64->flags);
    }
    MM_CUDA(cudaMemcpyAsync(h.data(), sb64->st, sizeof(CgState) * n_rhs, cudaMemcpyDeviceToHost, s));
    MM_CUDA(cudaStreamSynchronize(s));
    bool any_take = false;
    for (int k = 0; k < n_rhs; ++k) {
      take[k] = 0;
      if (inactive[k]) continue;
      total[k] += seg[k];
      I[k].fp32_applies += seg[k];
      if (!acc[k]) ++I[k].fp64_applies;
      ++I[k].outer_iters;
      if (R[k].status != 0) inner_status[k] = R[k].status;
      res[k] = acc[k] ? R[k].final_res : h[k].res / bnorm[k];
      if (res[k] < best[k]) {
        best[k] = res[k];
        best_iter[k] = total[k];
        take[k] = 1;
        any_take = true;
      }
      if (res[k] <= o.rel_tol || total[k] >= o.max_iter || seg[k] == 0) {
        inactive[k] = 1;
        --n_active;
      }
    }
    if (any_take) {
      // the flags buffer is reused for `take`; the next refinement step rewrites it
      MM_CUDA(cudaMemcpyAsync(sb64->flags, take.data(), sizeof(int) * n_rhs, cudaMemcpyHostToDevice, s));
      count_launches(1);
      k_take_best<<<gv, NT, 0, s>>>(sb64->x64, sb64->xbest64, nv, sb64->flags);
      MM_CUDA(cudaStreamSynchronize(s));
    }
    refine_ms += ms_since(t_ref);
  }
  write_hist(o, Hh, I);
  for (int k = 0; k < n_rhs; ++k) {
    I[k].t_pcg_ms = pcg_ms;
    I[k].t_refine_ms = refine_ms;
    I[k].iters = total[k];
    I[k].best_iter = best_iter[k];
    I[k].final_rel_res = res[k];
    I[k].best_rel_res = best[k];
    I[k].status = best[k] <= o.rel_tol ? MADMAP_OK : (inner_status[k] != 0 ? inner_status[k] : MADMAP_WARN_MAXITER);
  }
  *x_pad = sb64->xbest64;
  return MADMAP_OK;
}

static int worst_status(std::vector<madmap_solve_info>& I, double t_all) {
  int worst = MADMAP_OK;
  for (auto& x : I) {
    x.t_solve_ms = t_all;
    if (x.status < 0) worst = x.status;
    else if (worst == MADMAP_OK && x.status != MADMAP_OK) worst = x.status;
  }
  return worst;
}

template <int NS>
static madmap_status solve_impl(Plan* p, int n_rhs, const float* d, double* m, const madmap_solve_opts& o,
                                madmap_solve_info* info, cudaStream_t s) {
  auto t_start = std::chrono::steady_clock::now();
  Batch B;
  B.n_rhs = n_rhs;
  if (n_rhs > 1) {
    TileSet* ts = nullptr;
    madmap_status st = get_tile_set(p, n_rhs, &ts);
    if (st != MADMAP_OK) return st;
    B.ts = ts;
  }
  SolveBuffers* sb64 = nullptr;
  madmap_status st = get_buffers(p, true, n_rhs, &sb64);
  if (st != MADMAP_OK) return st;
  const long long nv = sb64->nvec;
  const int n = p->n_obs;
  std::vector<madmap_solve_info> I(n_rhs);
  for (auto& x : I) memset(&x, 0, sizeof(x));
  const bool fused = fused_residual(p, o);
  if (fused) {
    // b in float32: it only starts the first float32 inner solve (every
    // refinement residual is formed from d in full precision)
    SolveBuffers* sb32 = nullptr;
    st = get_buffers(p, false, n_rhs, &sb32);
    if (st != MADMAP_OK) return st;
    float* b32 = static_cast<float*>(sb32->q);
    MM_CUDA(cudaMemsetAsync(b32, 0, sizeof(float) * nv * n_rhs, s));
    if (B.ts)
      st = op_launch_set(p, OPP_F32, IN_TOD, OUT_MAP, d, b32, p->n_t, nv, nullptr, 0, B.ts, s);
    else
      st = op_launch(p, OPP_F32, IN_TOD, OUT_MAP, d, b32, 0, 0, 1, nullptr, s);
    if (st == MADMAP_OK) st = reduce_across(p, b32, nv * n_rhs, MADMAP_REDUCE_F32, s);
    if (st != MADMAP_OK) return st;
    count_launches(1);
    k_widen<<<grid_vec(nv * n_rhs), NT, 0, s>>>(b32, sb64->b64, nv * n_rhs);
  } else {
    // right-hand sides b = A^T N^-1 d into float64 maps (float64 or double-float arithmetic)
    MM_CUDA(cudaMemsetAsync(sb64->b64, 0, sizeof(double) * nv * n_rhs, s));
    if (B.ts)
      st = op_launch_set(p, refine_prec(o), IN_TOD, OUT_MAP, d, sb64->b64, p->n_t, nv, nullptr, 0, B.ts, s);
    else
      st = op_launch(p, refine_prec(o), IN_TOD, OUT_MAP, d, sb64->b64, 0, 0, 1, nullptr, s);
    if (st == MADMAP_OK) st = reduce_across(p, sb64->b64, nv * n_rhs, MADMAP_REDUCE_F64, s);
    if (st != MADMAP_OK) return st;
  }
  MM_CUDA(cudaStreamSynchronize(s));
  const double t_rhs =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  for (auto& x : I) {
    x.fp64_applies = fused ? 0 : 1;
    x.fp32_applies = fused ? 1 : 0;
    x.t_rhs_ms = t_rhs;
  }
  const double* xr = nullptr;
  st = solve_core<NS>(p, B, sb64, o, I, s, &xr, d);
  if (st != MADMAP_OK) return st;
  for (int k = 0; k < n_rhs; ++k) {
    count_launches(1);
    k_unpack<double, double><<<grid_vec((long long)n * p->n_stokes), NT, 0, s>>>(
        xr + k * nv, m + (long long)k * n * p->n_stokes, n, p->n_stokes, p->ns_pad);
  }
  MM_CUDA(cudaStreamSynchronize(s));
  MM_CUDA(cudaGetLastError());
  const double t_all = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  const int worst = worst_status(I, t_all);
  if (info) memcpy(info, I.data(), sizeof(madmap_solve_info) * n_rhs);
  return (madmap_status)worst;
}

// Continue a float64 solve from a checkpoint (single right-hand side).
template <int NS>
static madmap_status resume_impl(Plan* p, const madmap_checkpoint* c, double* m, const madmap_solve_opts& o,
                                 madmap_solve_info* info, cudaStream_t s) {
  auto t_start = std::chrono::steady_clock::now();
  Batch B;
  SolveBuffers* sb = nullptr;
  madmap_status st = get_buffers(p, true, 1, &sb);
  if (st != MADMAP_OK) return st;
  const int n = p->n_obs, ns = p->n_stokes, np = p->ns_pad;
  const long long user = (long long)n * ns;
  const double* src[5] = {c->x, c->r, c->z, c->p, c->x_best};
  double* dst[5] = {(double*)sb->x, (double*)sb->r, (double*)sb->z, (double*)sb->p, (double*)sb->xb};
  for (int k = 0; k < 5; ++k) {
    MM_CUDA(cudaMemcpyAsync(sb->b64, src[k], sizeof(double) * user, cudaMemcpyHostToDevice, s));
    count_launches(1);
    k_pack<double, double><<<grid_vec((long long)n * np), NT, 0, s>>>(sb->b64, dst[k], n, ns, np);
  }
  MM_CUDA(cudaMemsetAsync(sb->q, 0, sizeof(double) * sb->nvec, s));
  const int every = o.checkpoint_every > 0 ? o.checkpoint_every : 0;
  CgState h;
  memset(&h, 0, sizeof(h));
  h.rz = c->rz;
  h.bnorm = c->bnorm;
  h.res = c->rel_res;
  h.best_res = c->best_rel_res;
  h.tol = o.rel_tol;
  h.k = c->iters;
  h.best_k = c->best_iter;
  h.dir_k = c->iters;  // p already holds the next search direction
  h.max_iter = o.max_iter;
  h.done = (!(c->bnorm > 0.0) || c->rel_res <= o.rel_tol || c->iters >= o.max_iter) ? 1 : 0;
  h.pause_k = every ? c->iters + every : INT_MAX;
  h.halt = h.done;
  MM_CUDA(cudaMemcpyAsync(sb->st, &h, sizeof(CgState), cudaMemcpyHostToDevice, s));
  std::vector<PcgResult> R;
  int stopped = 0;
  const auto t_pcg = std::chrono::steady_clock::now();
  st = pcg64<NS>(p, sb, B, o, s, R, false, h.pause_k, &stopped);
  if (st != MADMAP_OK) return st;
  const double pcg_ms = ms_since(t_pcg);
  std::vector<std::vector<double>> Hh(1);
  if (o.residual_history && o.history_capacity > 0) {
    // iterations before the checkpoint were not seen by this call
    Hh[0].assign((size_t)std::min(c->iters, HIST_CAP), NAN);
    if (c->iters < HIST_CAP) Hh[0].push_back(c->rel_res);
    if ((st = append_hist(sb, 0, c->iters + 1, R[0].iters, 1.0, Hh[0], s)) != MADMAP_OK) return st;
  }
  count_launches(1);
  k_unpack<double, double><<<grid_vec(user), NT, 0, s>>>((const double*)sb->xb, m, n, ns, np);
  MM_CUDA(cudaStreamSynchronize(s));
  MM_CUDA(cudaGetLastError());
  std::vector<madmap_solve_info> Iv(1);
  memset(&Iv[0], 0, sizeof(Iv[0]));
  write_hist(o, Hh, Iv);
  madmap_solve_info& I = Iv[0];
  I.t_pcg_ms = pcg_ms;
  I.iters = R[0].iters;
  I.outer_iters = 1;
  I.best_iter = R[0].best_iter;
  I.fp64_applies = R[0].iters - c->iters;
  I.final_rel_res = R[0].final_res;
  I.best_rel_res = R[0].best_res;
  I.status = R[0].status != 0 ? R[0].status : (R[0].best_res <= o.rel_tol ? MADMAP_OK : MADMAP_WARN_MAXITER);
  if (stopped && I.status == MADMAP_WARN_MAXITER) I.status = MADMAP_STOPPED;
  I.t_solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  if (info) *info = I;
  return (madmap_status)I.status;
}

// ---------------------------------------------------------------- backward
// Gradients of a loss L(m) through the solve by the implicit adjoint: with
// lambda = H^-1 dL/dm (one more solve with the self-adjoint H),
//   dL/dd = N^-1 A lambda,
//   dL/df_k(tau) = sum over intervals of filter k of sum_{|t-t'| = tau}
//                  (A lambda)_t (d - A m)_t'   (both orders for tau > 0),
// from perturbing N^-1 and d in m = H^-1 A^T N^-1 d.

// out_t = alpha d_t + beta (A x)_t (float64 weights and map, float output);
// pix_pol (multi-resolution plans, else NULL) gives the Q/U slot of each sample
// (compressed pointing: ob.bore set, pix and cs unused)
// (extended pointing: ext gives the map row of each sample's extra column, or -1)
template <int NS>
__global__ void k_unpoint(const double* x, const int* pix, const int* pix_pol, const double2* cs, const float* d,
                          double alpha, double beta, float* out, long long n, const OtfPointing ob,
                          const int* ext, const int* hwp_base, const float* hwp_ang, const float* hwp_tau) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    float c2 = 0.f, s2 = 0.f;
    const int q = ob.bore ? otf_row(ob, t, NS == 3, c2, s2) : pix[t];
    double ax = 0.0;
    if (q >= 0) {
      if (NS == 1) {
        ax = x[q];
      } else {
        const double2 w = ob.bore ? make_double2(c2, s2) : cs[t];
        const int qp = pix_pol ? pix_pol[t] : q;
        ax = x[4LL * q] + x[4LL * qp + 1] * w.x + x[4LL * qp + 2] * w.y;
      }
      if (ext && ext[t] >= 0) ax += x[(long long)ext[t] * (NS == 1 ? 1 : 4)];
      if (hwp_base && hwp_base[t] >= 0) {
        double C[32];
        hwp_columns<double>(hwp_ang[t], hwp_tau[t], C);
        for (int i = 0; i < 32; ++i) ax += C[i] * x[(long long)(hwp_base[t] + i) * (NS == 1 ? 1 : 4)];
      }
    }
    out[t] = (float)((d ? alpha * (double)d[t] : 0.0) + beta * ax);
  }
}

// zero the adjoint right-hand side at unknowns without a row of H: excised
// pixels; excised_pol (multi-resolution plans, else NULL) covers the Q/U
// columns; rows from first_extra on (extended pointing) keep column 0 only
__global__ void k_mask_excised(double* b, long long nvec_pixels, int ns_pad, const unsigned char* excised,
                               const unsigned char* excised_pol, long long first_extra) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nvec_pixels * ns_pad;
       i += (long long)gridDim.x * blockDim.x) {
    const long long k = i / ns_pad;
    bool ex = (excised_pol && i % ns_pad != 0) ? excised_pol[k] : excised[k];
    if (k >= first_extra && i % ns_pad != 0) ex = true;
    if (ex) b[i] = 0.0;
  }
}

// Lag correlation sum_{|t-t'|=tau} a_t r_t' by direct sums: CTA (lag block,
// work item) covers CORR_LB lags over the samples [t_lo, t_hi) of one
// interval, in tiles of CORR_TT samples staged in shared memory, and adds
// its totals to grad[filter][tau] (float64 atomics, one per lag and item).
struct CorrItem {
  long long lo, hi;      // interval bounds
  long long t_lo, t_hi;  // samples of this item
  int filter, pad;
};

// Lag correlation sum_{t in item} a_t (r_{t+tau} + r_{t-tau}) (r outside the
// interval is 0; tau = 0 counts once).  Each thread owns CORR_R consecutive
// lags: per block of CORR_R samples it loads 2 CORR_R - 1 values of r per
// direction into registers and does CORR_R^2 multiply-adds per direction from
// them.  Shared r is padded one word per 8 so the threads' stride-8 reads hit
// distinct banks.  float32 products summed over a tile of CORR_TT samples,
// float64 across tiles and items.
constexpr int CORR_R = 8;
constexpr int CORR_T = 256;
constexpr int CORR_LB = CORR_R * CORR_T;  // lags per block
constexpr int CORR_TT = 1024;             // samples per tile
constexpr int CORR_W = CORR_TT + CORR_LB;
__device__ __forceinline__ int cpad(int i) { return i + (i >> 3); }

__global__ void __launch_bounds__(CORR_T) k_lag_corr(const float* a, const float* r, const CorrItem* items,
                                                    int n_lags, double* grad) {
  __shared__ float sa[CORR_TT];
  __shared__ float sp[CORR_W + CORR_W / 8];  // r[t0 + tau0 + i]
  __shared__ float sm[CORR_W + CORR_W / 8];  // r[t0 - tau0 - (CORR_LB - 1) + i]
  const CorrItem it = items[blockIdx.y];
  const int tau0 = blockIdx.x * CORR_LB;
  const int base = CORR_R * threadIdx.x;
  double tot[CORR_R];
#pragma unroll
  for (int j = 0; j < CORR_R; ++j) tot[j] = 0.0;
  for (long long t0 = it.t_lo; t0 < it.t_hi; t0 += CORR_TT) {
    const int nt = (int)min((long long)CORR_TT, it.t_hi - t0);
    __syncthreads();
    for (int k = threadIdx.x; k < CORR_TT; k += CORR_T) sa[k] = k < nt ? a[t0 + k] : 0.f;
    for (int i = threadIdx.x; i < CORR_W; i += CORR_T) {
      const long long tp = t0 + tau0 + i;
      const long long tm = t0 - tau0 - (CORR_LB - 1) + i;
      sp[cpad(i)] = (tp >= it.lo && tp < it.hi) ? r[tp] : 0.f;
      sm[cpad(i)] = (tm >= it.lo && tm < it.hi) ? r[tm] : 0.f;
    }
    __syncthreads();
    float acc1[CORR_R], acc2[CORR_R];
#pragma unroll
    for (int j = 0; j < CORR_R; ++j) acc1[j] = acc2[j] = 0.f;
    // samples past nt are zero in sa, so whole blocks of CORR_R are safe
    for (int k0 = 0; k0 < nt; k0 += CORR_R) {
      float v1[2 * CORR_R - 1], v2[2 * CORR_R - 1];
#pragma unroll
      for (int q = 0; q < 2 * CORR_R - 1; ++q) {
        v1[q] = sp[cpad(k0 + base + q)];
        v2[q] = sm[cpad(k0 + CORR_LB - CORR_R - base + q)];
      }
#pragma unroll
      for (int kk = 0; kk < CORR_R; ++kk) {
        const float ak = sa[k0 + kk];
#pragma unroll
        for (int j = 0; j < CORR_R; ++j) {
          acc1[j] = fmaf(ak, v1[kk + j], acc1[j]);
          acc2[j] = fmaf(ak, v2[kk - j + CORR_R - 1], acc2[j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < CORR_R; ++j) tot[j] += (double)acc1[j] + (tau0 + base + j == 0 ? 0.0 : (double)acc2[j]);
  }
#pragma unroll
  for (int j = 0; j < CORR_R; ++j) {
    const int tau = tau0 + base + j;
    if (tau < n_lags) atomicAdd(grad + (long long)it.filter * n_lags + tau, tot[j]);
  }
}

template <int NS>
static madmap_status backward_impl(Plan* p, const float* d, const double* m, const double* gm, float* grad_d,
                                   double* grad_lags, const madmap_solve_opts& o, madmap_solve_info* info,
                                   cudaStream_t s) {
  auto t_start = std::chrono::steady_clock::now();
  Batch B;
  SolveBuffers* sb64 = nullptr;
  madmap_status st = get_buffers(p, true, 1, &sb64);
  if (st != MADMAP_OK) return st;
  const long long nv = sb64->nvec;
  const int n = p->n_obs, ns = p->n_stokes, np = p->ns_pad;
  const long long nt = p->n_t;
  if (!p->bw_a) {
    st = dalloc_t(p, &p->bw_a, std::max(1LL, nt));
    if (st == MADMAP_OK) st = dalloc_t(p, &p->bw_r, std::max(1LL, nt));
    if (st != MADMAP_OK) return st;
  }
  // adjoint solve H lambda = dL/dm (zero at excised pixels)
  count_launches(2);
  k_pack<double, double><<<grid_vec(nv), NT, 0, s>>>(gm, sb64->b64, n, ns, np);
  k_mask_excised<<<grid_vec(nv), NT, 0, s>>>(sb64->b64, n, np, p->excised, p->multires ? p->excised_pol : nullptr,
                                             p->ext ? (long long)p->n_obs_sky : (long long)n);
  std::vector<madmap_solve_info> I(1);
  memset(&I[0], 0, sizeof(I[0]));
  const double* lam = nullptr;
  st = solve_core<NS>(p, B, sb64, o, I, s, &lam);
  if (st != MADMAP_OK) return st;
  // a = A lambda; r = d - A m  (m packed into the spare float64 vector t64)
  const int gt = (int)std::min<long long>((nt + 255) / 256, 152LL * 32);
  count_launches(3);
  const int* pix_pol = p->multires ? p->pix_obs_pol : nullptr;
  k_unpoint<NS><<<std::max(1, gt), 256, 0, s>>>(lam, p->pix_obs, pix_pol, p->cs64, nullptr, 0.0, 1.0, p->bw_a, nt,
                                                otf_pointing(p), p->ext_row, p->hwp_base, p->hwp_ang,
                                                p->hwp_tau);
  k_pack<double, double><<<grid_vec(nv), NT, 0, s>>>(m, sb64->t64, n, ns, np);
  k_unpoint<NS><<<std::max(1, gt), 256, 0, s>>>(sb64->t64, p->pix_obs, pix_pol, p->cs64, d, 1.0, -1.0, p->bw_r, nt,
                                                otf_pointing(p), p->ext_row, p->hwp_base, p->hwp_ang,
                                                p->hwp_tau);
  if (grad_d) {
    st = op_launch(p, false, IN_TOD_REAL, OUT_TOD, p->bw_a, grad_d, 0, 0, 1, nullptr, s);
    if (st != MADMAP_OK) return st;
  }
  if (grad_lags) {
    if (!p->corr_items) {
      std::vector<CorrItem> items;
      const long long chunk = 65536;
      for (int i = 0; i < p->n_ivl; ++i)
        for (long long t = p->offsets[i]; t < p->offsets[i + 1]; t += chunk)
          items.push_back({p->offsets[i], p->offsets[i + 1], t, std::min(p->offsets[i + 1], t + chunk),
                           p->ivl_filter[i], 0});
      p->n_corr_items = (int)items.size();
      CorrItem* dev = nullptr;
      st = dalloc(p, (void**)&dev, sizeof(CorrItem) * std::max<size_t>(1, items.size()));
      if (st != MADMAP_OK) return st;
      if (!items.empty())
        MM_CUDA(cudaMemcpy(dev, items.data(), sizeof(CorrItem) * items.size(), cudaMemcpyHostToDevice));
      p->corr_items = dev;
    }
    MM_CUDA(cudaMemsetAsync(grad_lags, 0, sizeof(double) * p->n_filters * p->n_lags, s));
    const CorrItem* items = static_cast<const CorrItem*>(p->corr_items);
    for (int y0 = 0; y0 < p->n_corr_items; y0 += 65535) {
      const int ny = std::min(65535, p->n_corr_items - y0);
      count_launches(1);
      k_lag_corr<<<dim3((p->n_lags + CORR_LB - 1) / CORR_LB, ny), CORR_T, 0, s>>>(p->bw_a, p->bw_r, items + y0,
                                                                                 p->n_lags, grad_lags);
    }
    st = reduce_across(p, grad_lags, (long long)p->n_filters * p->n_lags, MADMAP_REDUCE_F64, s);
    if (st != MADMAP_OK) return st;
  }
  MM_CUDA(cudaStreamSynchronize(s));
  MM_CUDA(cudaGetLastError());
  const double t_all = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  const int worst = worst_status(I, t_all);
  if (info) *info = I[0];
  return (madmap_status)worst;
}

// ---------------------------------------------------------------- operator entry points
template <typename Real>
static madmap_status apply_impl(Plan* p, int prec, int n_rhs, const void* x, void* y, cudaStream_t s) {
  SolveBuffers* sb = nullptr;
  madmap_status st = get_buffers(p, prec != OPP_F32, 1, &sb);
  if (st != MADMAP_OK) return st;
  const int n = p->n_obs, ns = p->n_stokes, np = p->ns_pad;
  const long long user = (long long)n * ns;
  for (int r = 0; r < n_rhs; ++r) {
    const Real* xr = static_cast<const Real*>(x) + r * user;
    Real* yr = static_cast<Real*>(y) + r * user;
    count_launches(2);
    k_pack<Real, Real><<<grid_vec((long long)n * np), NT, 0, s>>>(xr, (Real*)sb->p, n, ns, np);
    MM_CUDA(cudaMemsetAsync(sb->q, 0, sizeof(Real) * sb->nvec, s));
    const void* xin = sb->p;
    if (prec == OPP_DF64) {
      count_launches(1);
      k_split<<<grid_vec(sb->nvec), NT, 0, s>>>((const double*)sb->p, sb->xdf, sb->nvec);
      xin = sb->xdf;
    }
    st = op_launch(p, prec, IN_MAP, OUT_MAP, xin, sb->q, 0, 0, 1, nullptr, s);
    if (st == MADMAP_OK)
      st = reduce_across(p, sb->q, sb->nvec, prec == OPP_F32 ? MADMAP_REDUCE_F32 : MADMAP_REDUCE_F64, s);
    if (st != MADMAP_OK) return st;
    k_unpack<Real, Real><<<grid_vec(user), NT, 0, s>>>((const Real*)sb->q, yr, n, ns, np);
  }
  MM_CUDA(cudaGetLastError());
  return MADMAP_OK;
}

template <typename Real>
static madmap_status rhs_impl(Plan* p, int prec, int n_rhs, const float* d, void* b, cudaStream_t s) {
  SolveBuffers* sb = nullptr;
  madmap_status st = get_buffers(p, prec != OPP_F32, 1, &sb);
  if (st != MADMAP_OK) return st;
  const int n = p->n_obs, ns = p->n_stokes, np = p->ns_pad;
  const long long user = (long long)n * ns;
  for (int r = 0; r < n_rhs; ++r) {
    MM_CUDA(cudaMemsetAsync(sb->q, 0, sizeof(Real) * sb->nvec, s));
    st = op_launch(p, prec, IN_TOD, OUT_MAP, d + (long long)r * p->n_t, sb->q, 0, 0, 1, nullptr, s);
    if (st == MADMAP_OK)
      st = reduce_across(p, sb->q, sb->nvec, prec == OPP_F32 ? MADMAP_REDUCE_F32 : MADMAP_REDUCE_F64, s);
    if (st != MADMAP_OK) return st;
    count_launches(1);
    k_unpack<Real, Real><<<grid_vec(user), NT, 0, s>>>((const Real*)sb->q, static_cast<Real*>(b) + r * user, n, ns,
                                                       np);
  }
  MM_CUDA(cudaGetLastError());
  return MADMAP_OK;
}

}  // namespace mm

using namespace mm;

static madmap_status check_prec(int precision, bool allow_mixed, bool allow_df = false) {
  if (precision == MADMAP_FP64 || precision == MADMAP_FP32) return MADMAP_OK;
  if (allow_mixed && precision == MADMAP_MIXED) return MADMAP_OK;
  if (allow_df && precision == MADMAP_DF64) return MADMAP_OK;
  set_error("unsupported precision");
  return MADMAP_ERR_INVALID_ARG;
}
static int op_prec(int precision) {
  return precision == MADMAP_DF64 ? OPP_DF64 : precision == MADMAP_FP64 ? OPP_F64 : OPP_F32;
}

extern "C" madmap_status madmap_apply_ATNA(madmap_plan_t plan, int32_t precision, int32_t n_rhs, const void* x,
                                           void* y, void* stream) {
  MM_CHECK(plan && n_rhs >= 1, MADMAP_ERR_INVALID_ARG, "apply_ATNA: bad arguments");
  madmap_status st = check_prec(precision, false, true);
  if (st != MADMAP_OK) return st;
  Plan* p = reinterpret_cast<Plan*>(plan);
  MM_CHECK((x && y) || p->n_obs == 0, MADMAP_ERR_INVALID_ARG, "apply_ATNA: NULL map");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->n_obs == 0) return MADMAP_OK;
  return precision == MADMAP_FP32 ? apply_impl<float>(p, OPP_F32, n_rhs, x, y, s)
                                  : apply_impl<double>(p, op_prec(precision), n_rhs, x, y, s);
}

extern "C" madmap_status madmap_rhs(madmap_plan_t plan, int32_t precision, int32_t n_rhs, const float* d, void* b,
                                    void* stream) {
  MM_CHECK(plan && n_rhs >= 1, MADMAP_ERR_INVALID_ARG, "rhs: bad arguments");
  Plan* p = reinterpret_cast<Plan*>(plan);
  MM_CHECK(b || p->n_obs == 0, MADMAP_ERR_INVALID_ARG, "rhs: b is NULL");
  MM_CHECK(d || p->n_t == 0, MADMAP_ERR_INVALID_ARG, "rhs: d is NULL");
  madmap_status st = check_prec(precision, false, true);
  if (st != MADMAP_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->n_obs == 0) return MADMAP_OK;
  return precision == MADMAP_FP32 ? rhs_impl<float>(p, OPP_F32, n_rhs, d, b, s)
                                  : rhs_impl<double>(p, op_prec(precision), n_rhs, d, b, s);
}

extern "C" madmap_status madmap_apply_ninv(madmap_plan_t plan, int32_t precision, int32_t n_rhs, const void* y,
                                           void* w, void* stream) {
  MM_CHECK(plan && n_rhs >= 1, MADMAP_ERR_INVALID_ARG, "apply_ninv: bad arguments");
  Plan* p = reinterpret_cast<Plan*>(plan);
  MM_CHECK((y && w) || p->n_t == 0, MADMAP_ERR_INVALID_ARG, "apply_ninv: NULL timestream");
  madmap_status st = check_prec(precision, false);
  if (st != MADMAP_OK) return st;
  const bool fp64 = precision == MADMAP_FP64;
  const size_t es = fp64 ? sizeof(double) : sizeof(float);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int r = 0; r < n_rhs; ++r) {
    st = op_launch(p, fp64, IN_TOD_REAL, OUT_TOD, static_cast<const char*>(y) + (size_t)r * p->n_t * es,
                   static_cast<char*>(w) + (size_t)r * p->n_t * es, 0, 0, 1, nullptr, s);
    if (st != MADMAP_OK) return st;
  }
  return MADMAP_OK;
}

extern "C" void madmap_solve_opts_default(madmap_solve_opts* o) {
  if (!o) return;
  o->max_iter = 50;
  o->rel_tol = 1e-6;
  o->precision = MADMAP_FP64;
  o->max_outer = 10;
  o->inner_rel_tol = 1e-4;
  o->use_graph = 2;
  o->iters_per_sync = 8;
  o->refine_precision = MADMAP_DF64;
  o->checkpoint_every = 0;
  o->checkpoint = nullptr;
  o->on_checkpoint = nullptr;
  o->checkpoint_user = nullptr;
  o->residual_history = nullptr;
  o->history_capacity = 0;
  o->inner_restart = 0;
  o->final_residual = 0;
}

extern "C" madmap_status madmap_solve(madmap_plan_t plan, const float* d, double* m, const madmap_solve_opts* opts,
                                      madmap_solve_info* info, void* stream) {
  MM_CHECK(plan, MADMAP_ERR_INVALID_ARG, "solve: NULL plan");
  Plan* p = reinterpret_cast<Plan*>(plan);
  MM_CHECK(m || p->n_obs == 0, MADMAP_ERR_INVALID_ARG, "solve: m is NULL");
  MM_CHECK(d || p->n_t == 0, MADMAP_ERR_INVALID_ARG, "solve: d is NULL");
  madmap_solve_opts o;
  madmap_solve_opts_default(&o);
  if (opts) o = *opts;
  MM_CHECK(o.precision == MADMAP_FP64 || o.precision == MADMAP_MIXED, MADMAP_ERR_INVALID_ARG,
           "solve: precision must be FP64 or MIXED");
  MM_CHECK(o.checkpoint_every <= 0 || (o.precision == MADMAP_FP64 && o.checkpoint && o.checkpoint->x &&
                                       o.checkpoint->r && o.checkpoint->z && o.checkpoint->p && o.checkpoint->x_best),
           MADMAP_ERR_INVALID_ARG, "solve: checkpoints need precision FP64 and a checkpoint with five host maps");
  MM_CHECK(o.max_iter >= 0 && o.rel_tol >= 0 && o.iters_per_sync >= 1 && o.max_outer >= 1 &&
               o.inner_rel_tol > 0 && o.inner_rel_tol < 1 &&
               (o.refine_precision == MADMAP_DF64 || o.refine_precision == MADMAP_FP64),
           MADMAP_ERR_INVALID_ARG, "solve: bad options");
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  if (p->n_obs == 0) {
    if (info) {
      memset(info, 0, sizeof(*info));
    }
    return MADMAP_OK;
  }
  if (!p->solve_stream) {
    MM_CUDA(cudaStreamCreateWithFlags(&p->solve_stream, cudaStreamNonBlocking));
    MM_CUDA(cudaEventCreateWithFlags(&p->solve_event, cudaEventDisableTiming));
  }
  cudaStream_t s = p->solve_stream;
  MM_CUDA(cudaEventRecord(p->solve_event, caller));
  MM_CUDA(cudaStreamWaitEvent(s, p->solve_event, 0));
  madmap_status st = p->n_stokes == 1 ? solve_impl<1>(p, 1, d, m, o, info, s) : solve_impl<3>(p, 1, d, m, o, info, s);
  cudaStreamSynchronize(s);
  return st;
}

extern "C" madmap_status madmap_solve_resume(madmap_plan_t plan, const madmap_checkpoint* state, double* m,
                                             const madmap_solve_opts* opts, madmap_solve_info* info, void* stream) {
  MM_CHECK(plan && state, MADMAP_ERR_INVALID_ARG, "solve_resume: NULL plan or state");
  Plan* p = reinterpret_cast<Plan*>(plan);
  MM_CHECK(state->n_obs == p->n_obs && state->n_stokes == p->n_stokes, MADMAP_ERR_INVALID_ARG,
           "solve_resume: the state's map layout does not match the plan");
  MM_CHECK(p->n_obs == 0 || (m && state->x && state->r && state->z && state->p && state->x_best),
           MADMAP_ERR_INVALID_ARG, "solve_resume: NULL map");
  MM_CHECK(state->iters >= 0 && state->best_iter >= 0 && state->best_iter <= state->iters, MADMAP_ERR_INVALID_ARG,
           "solve_resume: bad iteration counts");
  madmap_solve_opts o;
  madmap_solve_opts_default(&o);
  if (opts) o = *opts;
  MM_CHECK(o.precision == MADMAP_FP64, MADMAP_ERR_INVALID_ARG, "solve_resume: precision must be FP64");
  MM_CHECK(o.max_iter >= 0 && o.rel_tol >= 0 && o.iters_per_sync >= 1, MADMAP_ERR_INVALID_ARG,
           "solve_resume: bad options");
  MM_CHECK(o.checkpoint_every <= 0 || (o.checkpoint && o.checkpoint->x && o.checkpoint->r && o.checkpoint->z &&
                                       o.checkpoint->p && o.checkpoint->x_best),
           MADMAP_ERR_INVALID_ARG, "solve_resume: checkpoints need a checkpoint with five host maps");
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  if (p->n_obs == 0) {
    if (info) memset(info, 0, sizeof(*info));
    return MADMAP_OK;
  }
  if (!p->solve_stream) {
    MM_CUDA(cudaStreamCreateWithFlags(&p->solve_stream, cudaStreamNonBlocking));
    MM_CUDA(cudaEventCreateWithFlags(&p->solve_event, cudaEventDisableTiming));
  }
  cudaStream_t s = p->solve_stream;
  MM_CUDA(cudaEventRecord(p->solve_event, caller));
  MM_CUDA(cudaStreamWaitEvent(s, p->solve_event, 0));
  madmap_status st = p->n_stokes == 1 ? resume_impl<1>(p, state, m, o, info, s) : resume_impl<3>(p, state, m, o, info, s);
  cudaStreamSynchronize(s);
  return st;
}

extern "C" madmap_status madmap_solve_backward(madmap_plan_t plan, const float* d, const double* m,
                                               const double* grad_m, float* grad_d, double* grad_lags,
                                               const madmap_solve_opts* opts, madmap_solve_info* info, void* stream) {
  MM_CHECK(plan, MADMAP_ERR_INVALID_ARG, "solve_backward: NULL plan");
  Plan* p = reinterpret_cast<Plan*>(plan);
  MM_CHECK((m && grad_m) || p->n_obs == 0, MADMAP_ERR_INVALID_ARG, "solve_backward: NULL map or map gradient");
  MM_CHECK(d || p->n_t == 0, MADMAP_ERR_INVALID_ARG, "solve_backward: d is NULL");
  madmap_solve_opts o;
  madmap_solve_opts_default(&o);
  if (opts) o = *opts;
  MM_CHECK(o.precision == MADMAP_FP64 || o.precision == MADMAP_MIXED, MADMAP_ERR_INVALID_ARG,
           "solve_backward: precision must be FP64 or MIXED");
  MM_CHECK(o.checkpoint_every <= 0, MADMAP_ERR_INVALID_ARG, "solve_backward: checkpoints are for forward solves");
  MM_CHECK(o.max_iter >= 0 && o.rel_tol >= 0 && o.iters_per_sync >= 1 && o.max_outer >= 1 &&
               o.inner_rel_tol > 0 && o.inner_rel_tol < 1 &&
               (o.refine_precision == MADMAP_DF64 || o.refine_precision == MADMAP_FP64),
           MADMAP_ERR_INVALID_ARG, "solve_backward: bad options");
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  if (p->n_obs == 0) {
    if (info) memset(info, 0, sizeof(*info));
    if (grad_lags) MM_CUDA(cudaMemsetAsync(grad_lags, 0, sizeof(double) * p->n_filters * p->n_lags, caller));
    if (grad_d && p->n_t) MM_CUDA(cudaMemsetAsync(grad_d, 0, sizeof(float) * p->n_t, caller));
    MM_CUDA(cudaStreamSynchronize(caller));
    return MADMAP_OK;
  }
  if (!p->solve_stream) {
    MM_CUDA(cudaStreamCreateWithFlags(&p->solve_stream, cudaStreamNonBlocking));
    MM_CUDA(cudaEventCreateWithFlags(&p->solve_event, cudaEventDisableTiming));
  }
  cudaStream_t s = p->solve_stream;
  MM_CUDA(cudaEventRecord(p->solve_event, caller));
  MM_CUDA(cudaStreamWaitEvent(s, p->solve_event, 0));
  madmap_status st = p->n_stokes == 1 ? backward_impl<1>(p, d, m, grad_m, grad_d, grad_lags, o, info, s)
                                      : backward_impl<3>(p, d, m, grad_m, grad_d, grad_lags, o, info, s);
  cudaStreamSynchronize(s);
  return st;
}

extern "C" madmap_status madmap_solve_batched(madmap_plan_t plan, int32_t n_rhs, const float* d, double* m,
                                              const madmap_solve_opts* opts, madmap_solve_info* info, void* stream) {
  MM_CHECK(plan && n_rhs >= 1, MADMAP_ERR_INVALID_ARG, "solve_batched: NULL plan or n_rhs < 1");
  Plan* p = reinterpret_cast<Plan*>(plan);
  MM_CHECK(m || p->n_obs == 0, MADMAP_ERR_INVALID_ARG, "solve_batched: m is NULL");
  MM_CHECK(d || p->n_t == 0, MADMAP_ERR_INVALID_ARG, "solve_batched: d is NULL");
  MM_CHECK(n_rhs <= 65535, MADMAP_ERR_INVALID_ARG, "solve_batched: at most 65535 right-hand sides");
  madmap_solve_opts o;
  madmap_solve_opts_default(&o);
  if (opts) o = *opts;
  MM_CHECK(o.precision == MADMAP_FP64 || o.precision == MADMAP_MIXED, MADMAP_ERR_INVALID_ARG,
           "solve_batched: precision must be FP64 or MIXED");
  MM_CHECK(o.checkpoint_every <= 0, MADMAP_ERR_INVALID_ARG, "solve_batched: checkpoints are for single solves");
  MM_CHECK(o.max_iter >= 0 && o.rel_tol >= 0 && o.iters_per_sync >= 1 && o.max_outer >= 1 &&
               o.inner_rel_tol > 0 && o.inner_rel_tol < 1 &&
               (o.refine_precision == MADMAP_DF64 || o.refine_precision == MADMAP_FP64),
           MADMAP_ERR_INVALID_ARG, "solve_batched: bad options");
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  if (p->n_obs == 0) {
    if (info) memset(info, 0, sizeof(*info) * n_rhs);
    return MADMAP_OK;
  }
  if (!p->solve_stream) {
    MM_CUDA(cudaStreamCreateWithFlags(&p->solve_stream, cudaStreamNonBlocking));
    MM_CUDA(cudaEventCreateWithFlags(&p->solve_event, cudaEventDisableTiming));
  }
  cudaStream_t s = p->solve_stream;
  MM_CUDA(cudaEventRecord(p->solve_event, caller));
  MM_CUDA(cudaStreamWaitEvent(s, p->solve_event, 0));
  madmap_status st = p->n_stokes == 1 ? solve_impl<1>(p, n_rhs, d, m, o, info, s)
                                      : solve_impl<3>(p, n_rhs, d, m, o, info, s);
  cudaStreamSynchronize(s);
  return st;
}

extern "C" madmap_status madmap_time_operator(madmap_plan_t plan, int32_t precision, int32_t reps, double* ms_out,
                                              int32_t* launches_out, void* stream) {
  MM_CHECK(plan && ms_out && reps >= 1, MADMAP_ERR_INVALID_ARG, "time_operator: bad arguments");
  MM_CHECK(precision == MADMAP_FP64 || precision == MADMAP_FP32 || precision == MADMAP_DF64, MADMAP_ERR_INVALID_ARG,
           "time_operator: precision must be FP64, FP32 or DF64");
  Plan* p = reinterpret_cast<Plan*>(plan);
  const int prec = op_prec(precision);
  SolveBuffers* sb = nullptr;
  madmap_status st = get_buffers(p, prec != OPP_F32, 1, &sb);
  if (st != MADMAP_OK) return st;
  int n_chunks, per_chunk;
  chunking(p, n_chunks, per_chunk);
  if (launches_out)
    for (int k = 0; k < 3; ++k) launches_out[k] = (p->diag && k > 0) ? 0 : n_chunks;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return op_time(p, prec, prec == OPP_DF64 ? (const void*)sb->xdf : sb->p, sb->q, reps, ms_out, s);
}
