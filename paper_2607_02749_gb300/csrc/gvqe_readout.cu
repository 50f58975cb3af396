// gvqe_readout.cu -- readout of a prepared state (Section IV-F, Section V-A):
// probabilities p(x) = |psi(x)|^2, the most probable bitstring, inverse-CDF
// shot sampling, and the CVaR-alpha of the outcome energy E(x) (Section III).
//
// Everything is summed in FP64 in fixed orders.  The CVaR search narrows the
// alpha-quantile of E with histograms whose bin masses are integer (p scaled
// by 2^60), so they do not depend on the order of the atomic adds.
#include <cstring>

#include "gvqe_engine.cuh"

namespace gvqe {
namespace {

constexpr int RO_NT = 256;

template <typename T>
__device__ __forceinline__ double prob(const T *psi, long long x) {
  const double v = (double)__ldcg(psi + x);
  return v * v;  // exact for an FP32 amplitude
}

// Order-preserving map of a double (given by its bits) onto an unsigned 64-bit
// key: comparisons of table energies run as integer compares (FP64 arithmetic
// is slow on this GPU).
__device__ __forceinline__ unsigned long long key_of_bits(unsigned long long b) {
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
// Keys (and bits) of the table entries 2i and 2i+1 (one 16-byte load).
__device__ __forceinline__ void key_pair(const double *E, long long i, unsigned long long &k0, unsigned long long &k1,
                                         unsigned long long &b0, unsigned long long &b1) {
  const longlong2 b = __ldcg(reinterpret_cast<const longlong2 *>(E) + i);
  b0 = (unsigned long long)b.x;
  b1 = (unsigned long long)b.y;
  k0 = key_of_bits(b0);
  k1 = key_of_bits(b1);
}
template <typename T>
__device__ __forceinline__ void amp_pair(const T *psi, long long i, T &v0, T &v1);
template <>
__device__ __forceinline__ void amp_pair<float>(const float *psi, long long i, float &v0, float &v1) {
  const float2 v = __ldcg(reinterpret_cast<const float2 *>(psi) + i);
  v0 = v.x;
  v1 = v.y;
}
template <>
__device__ __forceinline__ void amp_pair<double>(const double *psi, long long i, double &v0, double &v1) {
  const double2 v = __ldcg(reinterpret_cast<const double2 *>(psi) + i);
  v0 = v.x;
  v1 = v.y;
}

// Histogram mass of one amplitude, floor(p * 2^60): FP32 amplitudes square in
// FP32 and convert through the exponent and mantissa bits (integer work only);
// FP64 amplitudes square and convert in FP64.
__device__ __forceinline__ unsigned long long qmass(float v) {
  const float p = v * v;
  const unsigned b = __float_as_uint(p);
  const int ex = (int)((b >> 23) & 0xFF);
  const unsigned long long m = (b & 0x7FFFFFu) | (ex ? 0x800000u : 0u);
  const int sh = (ex ? ex : 1) - 90;  // p = m 2^(ex - 150); q = m 2^(ex - 90)
  return sh >= 0 ? (m << sh) : (sh > -64 ? (m >> -sh) : 0ull);
}
__device__ __forceinline__ unsigned long long qmass(double v) { return __double2ull_rz(v * v * 0x1p60); }

// Per chunk of 2^cb amplitudes: the sum of p (fixed tree order) and the first
// index of the chunk's largest p.
// A thread sums its (at most 32) p in the amplitude precision and compares
// |psi| (monotone in p, exact); the chunk sums above the thread are FP64.
template <typename T>
__global__ void __launch_bounds__(RO_NT) k_ro_chunks(const T *psi, int cb, double *csum, double *cmax,
                                                     long long *cidx) {
  __shared__ double ss[RO_NT], sm[RO_NT];
  __shared__ long long si[RO_NT];
  const long long c = blockIdx.x;
  const int tid = threadIdx.x;
  const long long base = c << cb;
  const int len = 1 << cb;
  T s = T(0), m = T(-1);
  long long mi = base;
  for (int i = tid; i < len; i += RO_NT) {
    const T v = __ldcg(psi + base + i);
    const T av = v < T(0) ? -v : v;
    s += v * v;
    if (av > m) {
      m = av;
      mi = base + i;
    }
  }
  ss[tid] = (double)s;
  sm[tid] = m < T(0) ? -1.0 : (double)m * (double)m;
  si[tid] = mi;
  __syncthreads();
  for (int w = RO_NT / 2; w > 0; w >>= 1) {
    if (tid < w) {
      ss[tid] += ss[tid + w];
      const double m2 = sm[tid + w];
      const long long i2 = si[tid + w];
      if (m2 > sm[tid] || (m2 == sm[tid] && i2 < si[tid])) {
        sm[tid] = m2;
        si[tid] = i2;
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    csum[c] = ss[0];
    cmax[c] = sm[0];
    cidx[c] = si[0];
  }
}

// One CTA: cdf[0] = 0, cdf[c + 1] = sum of chunks 0..c (block scans in a fixed
// order), the overall maximum (smallest index on ties) and the total.
__global__ void __launch_bounds__(1024) k_ro_scan(const double *csum, const double *cmax, const long long *cidx,
                                                  long long nch, double *cdf, double *stats, long long *argmax) {
  __shared__ double buf[1024];
  __shared__ double bm[1024];
  __shared__ long long bi[1024];
  const int tid = threadIdx.x;
  double carry = 0.0, m = -1.0;
  long long mi = 0;
  if (tid == 0) cdf[0] = 0.0;
  for (long long b0 = 0; b0 < nch; b0 += 1024) {
    const long long i = b0 + tid;
    double v = 0.0;
    if (i < nch) {
      v = csum[i];
      const double mm = cmax[i];
      const long long ii = cidx[i];
      if (mm > m || (mm == m && ii < mi)) {
        m = mm;
        mi = ii;
      }
    }
    buf[tid] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      const double add = tid >= off ? buf[tid - off] : 0.0;
      __syncthreads();
      buf[tid] += add;
      __syncthreads();
    }
    if (i < nch) cdf[i + 1] = carry + buf[tid];
    carry += buf[1023];
    __syncthreads();
  }
  bm[tid] = m;
  bi[tid] = mi;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (tid < w) {
      const double m2 = bm[tid + w];
      const long long i2 = bi[tid + w];
      if (m2 > bm[tid] || (m2 == bm[tid] && i2 < bi[tid])) {
        bm[tid] = m2;
        bi[tid] = i2;
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    stats[0] = bm[0];
    stats[2] = carry;
    argmax[0] = bi[0];
  }
}

// One warp per shot: t = u * total; the chunk whose cumulative range holds t
// (binary search), then a warp scan through that chunk for the first x whose
// cumulative probability exceeds t.  Where rounding leaves t past the chunk's
// own running sum, the chunk's last x with p > 0 is taken.
template <typename T>
__global__ void __launch_bounds__(RO_NT) k_ro_sample(const T *psi, int cb, long long nch, const double *cdf,
                                                     const double *u, int nshots, long long *shots) {
  const int lane = threadIdx.x & 31;
  const long long k = (blockIdx.x * (long long)RO_NT + threadIdx.x) >> 5;
  if (k >= nshots) return;  // the whole warp
  const double total = cdf[nch];
  double t = u[k] * total;
  if (!(t < total)) t = nextafter(total, 0.0);
  long long lo = 0, hi = nch - 1;  // first chunk c with cdf[c + 1] > t
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    if (cdf[mid + 1] > t)
      hi = mid;
    else
      lo = mid + 1;
  }
  const long long base = lo << cb;
  const int len = 1 << cb;
  double run = cdf[lo];
  long long found = -1, lastnz = -1;
  for (int i0 = 0; i0 < len; i0 += 32) {
    const int i = i0 + lane;
    const double p = i < len ? prob(psi, base + i) : 0.0;
    double incl = p;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const unsigned hit = __ballot_sync(0xffffffffu, p > 0.0 && run + incl > t);
    const unsigned nz = __ballot_sync(0xffffffffu, p > 0.0);
    if (nz) lastnz = base + i0 + 31 - __clz(nz);
    if (hit) {
      found = base + i0 + __ffs(hit) - 1;
      break;
    }
    run += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (found < 0) found = lastnz >= 0 ? lastnz : base;
  if (lane == 0) shots[k] = found;
}

// Keys of the smallest and largest E over all x: ext[1] (min), ext[2] (max).
__global__ void __launch_bounds__(RO_NT) k_ro_minmax(const double *E, long long N, unsigned long long *ext) {
  __shared__ unsigned long long smin, smax;
  if (threadIdx.x == 0) {
    smin = ~0ull;
    smax = 0ull;
  }
  __syncthreads();
  unsigned long long kmin = ~0ull, kmax = 0ull;
  const long long N2 = N >> 1, st = (long long)gridDim.x * RO_NT;
  for (long long i = blockIdx.x * (long long)RO_NT + threadIdx.x; i < N2; i += 2 * st) {
    unsigned long long k[4], raw[4];
    key_pair(E, i, k[0], k[1], raw[0], raw[1]);
    if (i + st < N2)
      key_pair(E, i + st, k[2], k[3], raw[2], raw[3]);
    else
      k[2] = k[3] = k[0];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      kmin = k[j] < kmin ? k[j] : kmin;
      kmax = k[j] > kmax ? k[j] : kmax;
    }
  }
  atomicMin(&smin, kmin);
  atomicMax(&smax, kmax);
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicMin(&ext[1], smin);
    atomicMax(&ext[2], smax);
  }
}

// One pass of the quantile search over the keys [edges[0], edges[RO_BINS]):
// the integer mass (p * 2^60) of every bin [edges[b], edges[b+1]) and the keys
// of the smallest and largest E inside the range (ext[1], ext[2]).  The edges
// are the keys of evenly spaced energies.  With `below` set, the masses under
// and above the range are summed too (ext[0], ext[3]); otherwise only x inside
// the range read their amplitude (the mass below is known from earlier passes).
//
// A key's bin: the range is cut into RO_LUT equal key intervals, lut[j] holds
// the bin of interval j's first key, so a key of interval j lies in a bin of
// [lut[j], lut[j+1]], found by a binary search over that (usually one- or
// two-bin) span instead of over all RO_BINS edges.
constexpr int RO_LUT_BITS = 11;
constexpr int RO_LUT = 1 << RO_LUT_BITS;
__device__ __forceinline__ int ro_bin_search(const unsigned long long *se, unsigned long long k, int b0, int b1) {
  while (b0 < b1) {  // largest b in [b0, b1] with se[b] <= k (se[b0] <= k holds)
    const int mid = (b0 + b1 + 1) >> 1;
    if (se[mid] <= k)
      b0 = mid;
    else
      b1 = mid - 1;
  }
  return b0;
}
template <typename T>
__global__ void __launch_bounds__(RO_NT) k_ro_hist(const T *psi, const double *E, long long N,
                                                   const unsigned long long *edges, unsigned long long *gmass,
                                                   unsigned long long *ext, int below) {
  __shared__ unsigned long long se[RO_BINS + 1];
  __shared__ unsigned long long sm[RO_BINS];
  __shared__ unsigned short lut[RO_LUT + 1];
  __shared__ unsigned long long smin, smax;
  for (int i = threadIdx.x; i <= RO_BINS; i += RO_NT) {
    se[i] = edges[i];
    if (i < RO_BINS) sm[i] = 0ull;
  }
  if (threadIdx.x == 0) {
    smin = ~0ull;
    smax = 0ull;
  }
  __syncthreads();
  const unsigned long long lo = se[0], hi = se[RO_BINS];
  const unsigned long long span = hi - lo;
  const int lsh = (span == 0ull) ? 0 : max(0, 64 - __clzll((long long)span) - RO_LUT_BITS);
  for (int j = threadIdx.x; j <= RO_LUT; j += RO_NT) {
    const unsigned long long kj = lo + ((unsigned long long)j << lsh);
    lut[j] = (unsigned short)((j == RO_LUT || kj >= hi || kj < lo) ? RO_BINS - 1 : ro_bin_search(se, kj, 0, RO_BINS - 1));
  }
  __syncthreads();
  const unsigned long long lo_read = below ? 0ull : lo;   // keys in [lo_read, hi_read) read psi
  const unsigned long long hi_read = below ? ~0ull : hi;
  unsigned long long kmin = ~0ull, kmax = 0ull, qbelow = 0ull, qabove = 0ull;
  auto add = [&](unsigned long long k, T v) {
    if (k < lo) {
      qbelow += qmass(v);
      return;
    }
    if (k >= hi) {
      qabove += qmass(v);
      return;
    }
    const unsigned long long q = qmass(v);
    const int j = (int)((k - lo) >> lsh);  // < RO_LUT
    const int b = ro_bin_search(se, k, lut[j], lut[j + 1]);  // largest b with edges[b] <= k
    if (q) atomicAdd(&sm[b], q);
    kmin = k < kmin ? k : kmin;
    kmax = k > kmax ? k : kmax;
  };
  const long long N2 = N >> 1, st = (long long)gridDim.x * RO_NT;
  for (long long i = blockIdx.x * (long long)RO_NT + threadIdx.x; i < N2; i += 2 * st) {
    unsigned long long k[4], raw[4];
    key_pair(E, i, k[0], k[1], raw[0], raw[1]);
    const bool two = i + st < N2;
    if (two) key_pair(E, i + st, k[2], k[3], raw[2], raw[3]);
    const bool in0 = k[0] >= lo_read && k[0] < hi_read, in1 = k[1] >= lo_read && k[1] < hi_read;
    const bool in2 = two && k[2] >= lo_read && k[2] < hi_read, in3 = two && k[3] >= lo_read && k[3] < hi_read;
    if (in0 || in1) {
      T v0, v1;
      amp_pair(psi, i, v0, v1);
      if (in0) add(k[0], v0);
      if (in1) add(k[1], v1);
    }
    if (in2 || in3) {
      T v2, v3;
      amp_pair(psi, i + st, v2, v3);
      if (in2) add(k[2], v2);
      if (in3) add(k[3], v3);
    }
  }
  atomicMin(&smin, kmin);
  atomicMax(&smax, kmax);
  if (qbelow) atomicAdd(&ext[0], qbelow);  // integer: order-independent
  if (qabove) atomicAdd(&ext[3], qabove);
  __syncthreads();
  for (int i = threadIdx.x; i < RO_BINS; i += RO_NT)
    if (sm[i]) atomicAdd(&gmass[i], sm[i]);
  if (threadIdx.x == 0) {
    atomicMin(&ext[1], smin);
    atomicMax(&ext[2], smax);
  }
}

// Energies at the shots, out[k] = E[shots[k]].
__global__ void k_ro_gather(const double *E, const long long *shots, int nshots, double *out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nshots) out[k] = E[shots[k]];
}

// Tail sums for the CVaR: per CTA sum of p*E and p over E < tau, and of p over
// E == tau (fixed per-thread order, fixed tree).
// Compensated (Kahan) running sum in the amplitude precision: FP32 amplitudes
// keep the tail sums off the (slow) FP64 pipe; FP64 amplitudes sum in FP64.
template <typename T>
struct KSum {
  T s = T(0), c = T(0);
  __device__ __forceinline__ void add(T x) {
    const T y = x - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

template <typename T>
__global__ void __launch_bounds__(RO_NT) k_ro_tail(const T *psi, const double *E, long long N,
                                                   unsigned long long ktau, double *part) {
  __shared__ double r[3][RO_NT];
  KSum<T> ksb, kpb, kpa;
  auto add = [&](unsigned long long k, T v, unsigned long long bits) {
    const T p = v * v;
    if (k < ktau) {
      ksb.add(p * (T)__longlong_as_double((long long)bits));
      kpb.add(p);
    } else {
      kpa.add(p);
    }
  };
  const long long N2 = N >> 1, st = (long long)gridDim.x * RO_NT;
  for (long long i = blockIdx.x * (long long)RO_NT + threadIdx.x; i < N2; i += 2 * st) {
    unsigned long long k[4], raw[4];
    key_pair(E, i, k[0], k[1], raw[0], raw[1]);
    const bool two = i + st < N2;
    if (two) key_pair(E, i + st, k[2], k[3], raw[2], raw[3]);
    if (k[0] <= ktau || k[1] <= ktau) {
      T v0, v1;
      amp_pair(psi, i, v0, v1);
      if (k[0] <= ktau) add(k[0], v0, raw[0]);
      if (k[1] <= ktau) add(k[1], v1, raw[1]);
    }
    if (two && (k[2] <= ktau || k[3] <= ktau)) {
      T v2, v3;
      amp_pair(psi, i + st, v2, v3);
      if (k[2] <= ktau) add(k[2], v2, raw[2]);
      if (k[3] <= ktau) add(k[3], v3, raw[3]);
    }
  }
  const int tid = threadIdx.x;
  r[0][tid] = (double)ksb.s - (double)ksb.c;
  r[1][tid] = (double)kpb.s - (double)kpb.c;
  r[2][tid] = (double)kpa.s - (double)kpa.c;
  __syncthreads();
  for (int w = RO_NT / 2; w > 0; w >>= 1) {
    if (tid < w)
      for (int j = 0; j < 3; ++j) r[j][tid] += r[j][tid + w];
    __syncthreads();
  }
  if (tid < 3) part[3 * (long long)blockIdx.x + tid] = r[tid][0];
}

// CVaR_alpha = (S + clamp(alpha T - P, 0, Pa) tau) / (alpha T), T = stats[2]:
// the lowest-energy alpha fraction of the outcomes, the outcomes at E == tau
// counted for the remainder.
__global__ void k_ro_cvar(const double *part, int nparts, double alpha, double tau, double *stats) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double S = 0.0, P = 0.0, Pa = 0.0;
  for (int i = 0; i < nparts; ++i) {
    S += part[3 * i];
    P += part[3 * i + 1];
    Pa += part[3 * i + 2];
  }
  const double aT = alpha * stats[2];
  double rest = aT - P;
  rest = rest < 0.0 ? 0.0 : (rest > Pa ? Pa : rest);
  stats[1] = (S + rest * tau) / aT;
}

inline int ro_grid() { return num_sms_cached() * 4; }

}  // namespace

int readout_chunk_bits(int n) { return n < 13 ? n : 13; }
int readout_tail_parts() { return ro_grid(); }

// Complex path: out[x] = |psi(x)| from interleaved (re, im) amplitudes.
template <typename T>
__global__ void k_ro_modulus(const T *__restrict__ psi, long long N, T *__restrict__ out) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < N; x += (long long)gridDim.x * blockDim.x) {
    const T re = __ldcg(psi + 2 * x), im = __ldcg(psi + 2 * x + 1);
    out[x] = sqrt(re * re + im * im);
  }
}

cudaError_t launch_ro_modulus(int prec, const void *psi, int n, void *out, cudaStream_t s) {
  const long long N = 1LL << n;
  const long long blocks = (N + RO_NT - 1) / RO_NT;
  const unsigned g = (unsigned)(blocks < 65536 ? blocks : 65536);
  if (prec)
    k_ro_modulus<double><<<g, RO_NT, 0, s>>>((const double *)psi, N, (double *)out);
  else
    k_ro_modulus<float><<<g, RO_NT, 0, s>>>((const float *)psi, N, (float *)out);
  return cudaGetLastError();
}

cudaError_t launch_ro_prob(int prec, const void *psi, int n, double *csum, double *cmax, long long *cidx,
                           double *cdf, double *stats, long long *argmax, cudaStream_t s) {
  const int cb = readout_chunk_bits(n);
  const long long nch = 1LL << (n - cb);
  if (prec)
    k_ro_chunks<double><<<(unsigned)nch, RO_NT, 0, s>>>((const double *)psi, cb, csum, cmax, cidx);
  else
    k_ro_chunks<float><<<(unsigned)nch, RO_NT, 0, s>>>((const float *)psi, cb, csum, cmax, cidx);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_ro_scan<<<1, 1024, 0, s>>>(csum, cmax, cidx, nch, cdf, stats, argmax);
  return cudaGetLastError();
}

cudaError_t launch_ro_sample(int prec, const void *psi, int n, const double *cdf, const double *u, int nshots,
                             long long *shots, cudaStream_t s) {
  if (nshots <= 0) return cudaSuccess;
  const int cb = readout_chunk_bits(n);
  const long long nch = 1LL << (n - cb);
  const unsigned grid = (unsigned)(((long long)nshots * 32 + RO_NT - 1) / RO_NT);
  if (prec)
    k_ro_sample<double><<<grid, RO_NT, 0, s>>>((const double *)psi, cb, nch, cdf, u, nshots, shots);
  else
    k_ro_sample<float><<<grid, RO_NT, 0, s>>>((const float *)psi, cb, nch, cdf, u, nshots, shots);
  return cudaGetLastError();
}

cudaError_t launch_ro_minmax(const double *E, int n, unsigned long long *ext, cudaStream_t s) {
  k_ro_minmax<<<ro_grid(), RO_NT, 0, s>>>(E, 1LL << n, ext);
  return cudaGetLastError();
}

cudaError_t launch_ro_hist(int prec, const void *psi, const double *E, int n, const unsigned long long *edges,
                           unsigned long long *gmass, unsigned long long *ext, int below, cudaStream_t s) {
  if (prec)
    k_ro_hist<double><<<ro_grid(), RO_NT, 0, s>>>((const double *)psi, E, 1LL << n, edges, gmass, ext, below);
  else
    k_ro_hist<float><<<ro_grid(), RO_NT, 0, s>>>((const float *)psi, E, 1LL << n, edges, gmass, ext, below);
  return cudaGetLastError();
}

cudaError_t launch_ro_gather(const double *E, const long long *shots, int nshots, double *out, cudaStream_t s) {
  if (nshots <= 0) return cudaSuccess;
  k_ro_gather<<<(nshots + 255) / 256, 256, 0, s>>>(E, shots, nshots, out);
  return cudaGetLastError();
}

cudaError_t launch_ro_cvar(int prec, const void *psi, const double *E, int n, double alpha, double tau,
                           double *part, double *stats, cudaStream_t s) {
  const int g = ro_grid();
  unsigned long long kt;
  memcpy(&kt, &tau, sizeof(kt));
  kt = (kt >> 63) ? ~kt : (kt | 0x8000000000000000ull);
  if (prec)
    k_ro_tail<double><<<g, RO_NT, 0, s>>>((const double *)psi, E, 1LL << n, kt, part);
  else
    k_ro_tail<float><<<g, RO_NT, 0, s>>>((const float *)psi, E, 1LL << n, kt, part);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_ro_cvar<<<1, 32, 0, s>>>(part, g, alpha, tau, stats);
  return cudaGetLastError();
}

}  // namespace gvqe
