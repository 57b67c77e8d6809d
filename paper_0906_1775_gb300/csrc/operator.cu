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
#include "internal.cuh"

namespace mm {

namespace {

enum { IN_MAPX = 0, IN_TODF = 1, IN_TODR = 2 };

struct OpArgs {
  const Tile* tiles;
  int tile0;
  int M, N1, N2, logN1, logN2, B1, logB1, B2;
  const int* pix;
  const float* psi;
  const double2* cs64;
  const void* in;
  long long in_stride;
  void* out;
  long long out_stride;
  void* scratch;
  const void* H;
  const void* tw;
  const int* skip;
};

template <typename Real>
__device__ __forceinline__ void weights(const OpArgs& a, long long t, Real& c, Real& s);
template <>
__device__ __forceinline__ void weights<float>(const OpArgs& a, long long t, float& c, float& s) {
  sincosf(2.0f * a.psi[t], &s, &c);
}
template <>
__device__ __forceinline__ void weights<double>(const OpArgs& a, long long t, double& c, double& s) {
  const double2 cs = a.cs64[t];
  c = cs.x;
  s = cs.y;
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

template <typename Real, int NS>
__device__ __forceinline__ void scatter(Real* y, int p, Real v, Real c, Real s);
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

template <typename Real, int NS, int IN>
__device__ __forceinline__ Real load_sample(const OpArgs& a, const Lane& L, int n) {
  const long long t = L.ws + n;
  if (t < L.lo || t >= L.hi) return Real(0);
  if (IN == IN_TODF) return (Real)(static_cast<const float*>(a.in)[L.rhs * a.in_stride + t]);
  if (IN == IN_TODR) return static_cast<const Real*>(a.in)[L.rhs * a.in_stride + t];
  const int p = a.pix[t];
  if (p < 0) return Real(0);
  Real c = 0, s = 0;
  if (NS == 3) weights<Real>(a, t, c, s);
  return gather<Real, NS>(static_cast<const Real*>(a.in) + L.rhs * a.in_stride, p, c, s);
}

template <typename Real, int NS, int OUT>
__device__ __forceinline__ void emit_sample(const OpArgs& a, const Lane& L, int n, Real v) {
  if (n < L.out_lo || n >= L.out_hi) return;
  const long long t = L.ws + n;
  if (OUT == OUT_TOD) {
    static_cast<Real*>(a.out)[L.rhs * a.out_stride + t] = v;
    return;
  }
  const int p = a.pix[t];
  if (p < 0) return;
  Real c = 0, s = 0;
  if (NS == 3) weights<Real>(a, t, c, s);
  scatter<Real, NS>(static_cast<Real*>(a.out) + L.rhs * a.out_stride, p, v, c, s);
}

__device__ __forceinline__ Lane load_lane(const Lane& g) {
  Lane L;
  L.ws = g.ws;
  L.lo = g.lo;
  L.hi = g.hi;
  L.out_lo = g.out_lo;
  L.out_hi = g.out_hi;
  L.rhs = g.rhs;
  L.pad = 0;
  return L;
}

// ---------------------------------------------------------------- k_f1
template <typename Real, int NS, int IN>
__global__ void __launch_bounds__(256) k_f1(OpArgs a) {
  typedef typename CxT<Real>::type C;
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int rs = row_stride(a.N2);
  C* tw = buf + a.B1 * rs;
  const C* twM = static_cast<const C*>(a.tw);
  for (int k = threadIdx.x; k < (a.N2 >> 1); k += blockDim.x) tw[k] = twM[(long long)k * a.N1];
  const int tl = blockIdx.y;
  const Tile* T = a.tiles + a.tile0 + tl;
  const Lane L0 = load_lane(T->l[0]);
  const Lane L1 = load_lane(T->l[1]);
  const int n1_0 = blockIdx.x * a.B1;
  const int total = a.B1 << a.logN2;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int j = e & (a.B1 - 1);
    const int n2 = e >> a.logB1;
    const int n = n1_0 + j + (n2 << a.logN1);
    C v;
    v.x = load_sample<Real, NS, IN>(a, L0, n);
    v.y = load_sample<Real, NS, IN>(a, L1, n);
    buf[j * rs + sidx(n2)] = v;
  }
  __syncthreads();
  fft_rows<C, false>(buf, a.B1, rs, a.logN2, tw);
  C* sc = static_cast<C*>(a.scratch) + (long long)tl * a.M;
  const int mask = a.M - 1;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int j = e & (a.B1 - 1);
    const int pos = e >> a.logB1;
    const int n1 = n1_0 + j;
    const int k2 = brev_n(pos, a.logN2);
    sc[(long long)pos * a.N1 + n1] = cmul(buf[j * rs + sidx(pos)], twM[(n1 * k2) & mask]);
  }
}

// ---------------------------------------------------------------- k_f2
template <typename Real>
__global__ void __launch_bounds__(256) k_f2(OpArgs a) {
  typedef typename CxT<Real>::type C;
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int rs = row_stride(a.N1);
  C* tw = buf + a.B2 * rs;
  const C* twM = static_cast<const C*>(a.tw);
  for (int k = threadIdx.x; k < (a.N1 >> 1); k += blockDim.x) tw[k] = twM[(long long)k * a.N2];
  const int tl = blockIdx.y;
  const Tile* T = a.tiles + a.tile0 + tl;
  const int filt = T->filter;
  const int pos0 = blockIdx.x * a.B2;
  C* sc = static_cast<C*>(a.scratch) + (long long)tl * a.M + (long long)pos0 * a.N1;
  const int total = a.B2 << a.logN1;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int i = e >> a.logN1;
    const int n1 = e & (a.N1 - 1);
    buf[i * rs + sidx(n1)] = sc[e];
  }
  __syncthreads();
  fft_rows<C, false>(buf, a.B2, rs, a.logN1, tw);
  const Real* H = static_cast<const Real*>(a.H) + (long long)filt * a.M + (long long)pos0 * a.N1;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int i = e >> a.logN1;
    const int p1 = e & (a.N1 - 1);
    const Real h = H[e];
    C& z = buf[i * rs + sidx(p1)];
    z.x *= h;
    z.y *= h;
  }
  __syncthreads();
  fft_rows<C, true>(buf, a.B2, rs, a.logN1, tw);
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int i = e >> a.logN1;
    const int n1 = e & (a.N1 - 1);
    sc[e] = buf[i * rs + sidx(n1)];
  }
}

// ---------------------------------------------------------------- k_f3
template <typename Real, int NS, int OUT>
__global__ void __launch_bounds__(256) k_f3(OpArgs a) {
  typedef typename CxT<Real>::type C;
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int rs = row_stride(a.N2);
  C* tw = buf + a.B1 * rs;
  const C* twM = static_cast<const C*>(a.tw);
  for (int k = threadIdx.x; k < (a.N2 >> 1); k += blockDim.x) tw[k] = twM[(long long)k * a.N1];
  const int tl = blockIdx.y;
  const Tile* T = a.tiles + a.tile0 + tl;
  const Lane L0 = load_lane(T->l[0]);
  const Lane L1 = load_lane(T->l[1]);
  const int n1_0 = blockIdx.x * a.B1;
  const int total = a.B1 << a.logN2;
  const C* sc = static_cast<const C*>(a.scratch) + (long long)tl * a.M;
  const int mask = a.M - 1;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int j = e & (a.B1 - 1);
    const int pos = e >> a.logB1;
    const int n1 = n1_0 + j;
    const int k2 = brev_n(pos, a.logN2);
    buf[j * rs + sidx(pos)] = cmulc(sc[(long long)pos * a.N1 + n1], twM[(n1 * k2) & mask]);
  }
  __syncthreads();
  fft_rows<C, true>(buf, a.B1, rs, a.logN2, tw);
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int j = e & (a.B1 - 1);
    const int n2 = e >> a.logB1;
    const int n = n1_0 + j + (n2 << a.logN1);
    const C v = buf[j * rs + sidx(n2)];
    emit_sample<Real, NS, OUT>(a, L0, n, v.x);
    emit_sample<Real, NS, OUT>(a, L1, n, v.y);
  }
}

template <typename Real>
inline int elems_per_cta() {
  return sizeof(Real) == 4 ? 8192 : 4096;
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
  return (size_t)(B1 * row_stride(p->N2) + (p->N2 >> 1)) * sizeof(typename CxT<Real>::type);
}
template <typename Real>
size_t smem_f2(const Plan* p) {
  int B1, B2;
  geometry<Real>(p, B1, B2);
  return (size_t)(B2 * row_stride(p->N1) + (p->N1 >> 1)) * sizeof(typename CxT<Real>::type);
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename Real, int NS, int IN, int OUT>
madmap_status launch_all(Plan* p, const void* in, void* out, long long in_stride, long long out_stride,
                         int n_rhs, const int* skip, cudaStream_t s) {
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
  a.scratch = p->scratch;
  a.H = sizeof(Real) == 8 ? (const void*)p->H64 : (const void*)p->H32;
  a.tw = sizeof(Real) == 8 ? (const void*)p->tw64 : (const void*)p->tw32;
  a.skip = skip;
  a.tiles = p->tiles;
  const size_t sm13 = smem_f13<Real>(p), sm2 = smem_f2<Real>(p);
  // opt-in to large dynamic shared memory once per kernel instance (raised when
  // a plan needs more); n_rhs == 0 only does this, so it can precede a capture
  static size_t set13 = 0, set2 = 0;
  if (sm13 > set13) {
    MM_CUDA(set_smem(k_f1<Real, NS, IN>, sm13));
    MM_CUDA(set_smem(k_f3<Real, NS, OUT>, sm13));
    set13 = sm13;
  }
  if (sm2 > set2) {
    MM_CUDA(set_smem(k_f2<Real>, sm2));
    set2 = sm2;
  }
  for (int r = 0; r < n_rhs; ++r) {
    a.in = static_cast<const char*>(in) + (size_t)r * in_stride *
                                              (IN == IN_TODF ? sizeof(float) : sizeof(Real));
    a.out = static_cast<char*>(out) + (size_t)r * out_stride * sizeof(Real);
    a.in_stride = 0;
    a.out_stride = 0;
    for (int t0 = 0; t0 < p->n_tiles; t0 += p->tiles_per_chunk) {
      const int nt = (p->n_tiles - t0) < p->tiles_per_chunk ? (p->n_tiles - t0) : p->tiles_per_chunk;
      a.tile0 = t0;
      dim3 g13(p->N1 / a.B1, nt), g2(p->N2 / a.B2, nt);
      k_f1<Real, NS, IN><<<g13, 256, sm13, s>>>(a);
      k_f2<Real><<<g2, 256, sm2, s>>>(a);
      k_f3<Real, NS, OUT><<<g13, 256, sm13, s>>>(a);
    }
  }
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
  if (in_mode == IN_TOD_REAL && out_mode == OUT_TOD)
    return launch_all<Real, NS, IN_TODR, OUT_TOD>(p, in, out, is, os, n_rhs, skip, s);
  if (in_mode == IN_MAP && out_mode == OUT_TOD)
    return launch_all<Real, NS, IN_MAPX, OUT_TOD>(p, in, out, is, os, n_rhs, skip, s);
  set_error("unsupported operator mode");
  return MADMAP_ERR_INTERNAL;
}

}  // namespace

size_t f1_smem_bytes(const Plan* p, bool fp64) {
  return fp64 ? smem_f13<double>(p) : smem_f13<float>(p);
}

// in_mode: IN_MAP (gather from a map), IN_TOD (float timestream, e.g. the
// data d) or IN_TOD_REAL (timestream of the working precision).  n_rhs == 0
// only prepares the kernels (shared-memory opt-in) and launches nothing.
madmap_status op_launch(Plan* p, bool fp64, int in_mode, int out_mode, const void* in, void* out,
                        long long in_stride, long long out_stride, int n_rhs, const int* skip,
                        cudaStream_t s) {
  if (p->n_tiles == 0) return MADMAP_OK;
  if (fp64) {
    if (p->n_stokes == 1)
      return dispatch_io<double, 1>(p, in_mode, out_mode, in, out, in_stride, out_stride, n_rhs, skip, s);
    return dispatch_io<double, 3>(p, in_mode, out_mode, in, out, in_stride, out_stride, n_rhs, skip, s);
  }
  if (p->n_stokes == 1)
    return dispatch_io<float, 1>(p, in_mode, out_mode, in, out, in_stride, out_stride, n_rhs, skip, s);
  return dispatch_io<float, 3>(p, in_mode, out_mode, in, out, in_stride, out_stride, n_rhs, skip, s);
}

}  // namespace mm
