// gvqe_kernels.cu -- dispatcher, whole-register kernel and support kernels of
// the gvqe engine.  The tile-pass kernels (tile bits >= 10) are templates in
// gvqe_tile.cuh, instantiated by gvqe_inst.cu once per (type, tile bits).
#include <cstdio>

#include "gvqe_engine.cuh"

namespace gvqe {

template <typename T, int TB>
cudaError_t launch_tb(const PassArgs &A, int jobs, int nterm, cudaStream_t s);

namespace {

template <typename T>
struct V2;
template <>
struct V2<float> {
  using type = float2;
};
template <>
struct V2<double> {
  using type = double2;
};


template <typename T, typename T2>
__device__ __forceinline__ T product_state(long long x, const T2 *l0, int n) {
  T p = T(1);
  for (int q = 0; q < n; ++q) p *= ((x >> q) & 1) ? l0[q].y : l0[q].x;
  return p;
}

template <typename T, typename T2>
__device__ __forceinline__ T load_val(int mode, const T *__restrict__ in, long long y, long long nmask,
                                      const T2 *l0, int n, const EntMap &ent) {
  switch (mode) {
    case LD_ZERO:
      return y == 0 ? T(1) : T(0);
    case LD_GATHER:
      return in[ent_inv((uint32_t)y, (uint32_t)nmask, ent, n)];
    case LD_L0_GATHER:
      return product_state<T>(ent_inv((uint32_t)y, (uint32_t)nmask, ent, n), l0, n);
    case LD_L0:
      return product_state<T>(y, l0, n);
    default:
      return in[y];
  }
}

template <typename T>
__device__ __forceinline__ void store_val(int mode, T *__restrict__ out, long long y, long long nmask, T v, int n,
                                          const EntMap &ent) {
  if (mode == ST_PLAIN)
    out[y] = v;
  else if (mode == ST_SCATTER)
    out[ent_inv((uint32_t)y, (uint32_t)nmask, ent, n)] = v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T2>
__device__ __forceinline__ void load_coeffs(const PassArgs &A, const T2 *cs, T2 *gcs, T2 *l0cs, int tid) {
  if (tid < 16) {
    T2 v;
    v.x = 1;
    v.y = 0;
    if (tid < A.tb && ((A.gate_mask >> tid) & 1u) && A.kind != K_WHT) {
      const int q = tile_gbit(tid, A.c, A.a, A.k1, A.gap);
      v = cs[A.layer * A.pstride + q - A.qoff];
    }
    gcs[tid] = v;
  }
  if (tid < 32 && tid < A.n && l0cs != nullptr &&
      (A.load_mode == LD_L0 || A.load_mode == LD_L0_GATHER || A.kind == K_GRAD_L0))
    l0cs[tid] = cs[tid];
}

// --------------------------------------------- whole-register kernel (n < 10) --
// One CTA per job holds the whole state (2^n <= 512 amplitudes) and applies
// the pass one gate bit at a time.  Reductions are per-thread FP64 partials
// summed in thread order.
constexpr int SMALL_NT = 128;
constexpr int SMALL_MAXN = 9;

// The complex path (F_COMPLEX): index bit 0 is the re/im channel (no gate); a
// pass's RZ gates follow its RY gates as one phase per amplitude, the backward
// pass takes RZ gradients Im<lam|Z|psi>, corrects the RY gradients to
// cos(tz) Y - sin(tz) X and un-applies the phase before the RY rotations.
template <typename T, typename T2>
__device__ __forceinline__ T2 small_phase(int x, uint32_t gm, int n, const T2 *zcs) {
  T2 p;
  p.x = 1;
  p.y = 0;
  for (int b = 1; b < n; ++b) {
    if (!((gm >> b) & 1u)) continue;
    T2 e = zcs[b];
    if (!((x >> b) & 1)) e.y = -e.y;  // x_q = 0: exp(-i theta/2)
    const T re = p.x * e.x - p.y * e.y;
    p.y = p.x * e.y + p.y * e.x;
    p.x = re;
  }
  return p;
}

template <typename T>
__global__ void __launch_bounds__(SMALL_NT) k_small(const PassArgs A) {
  using T2 = typename V2<T>::type;
  constexpr int ES = 2 * SMALL_MAXN;  // energy slot; RY rows 0..8, RZ rows 9..17
  __shared__ T sp[1 << SMALL_MAXN], sl[1 << SMALL_MAXN];
  __shared__ T2 gcs[16];
  __shared__ T2 zcs[16];
  __shared__ T2 l0cs[32];
  __shared__ double red[SMALL_NT][ES + 1];
  const int job = blockIdx.y;
  const int tid = threadIdx.x;
  const int n = A.n;
  const int N = 1 << n;
  const long long nmask = N - 1;
  if (A.minlayer != nullptr && !(A.flags & F_ENERGY)) {
    if (A.kind == K_BWD && A.layer < A.minlayer[A.job0 + job]) return;
    if (A.kind == K_GRAD_L0 && A.minlayer[A.job0 + job] > 0) return;
  }
  const T2 *cs = reinterpret_cast<const T2 *>(A.cs) + (size_t)(A.job0 + job) * A.P;
  const bool cplx = (A.flags & F_COMPLEX) != 0;
  if (A.kind != K_WHT) load_coeffs(A, cs, gcs, l0cs, tid);
  if (cplx && tid < 16) {
    T2 v;
    v.x = 1;
    v.y = 0;
    if (tid < A.tb && ((A.gate_mask >> tid) & 1u)) v = cs[A.layer * A.pstride + A.zoff + tid - A.qoff];
    zcs[tid] = v;
  }
  __syncthreads();
  const T *in = reinterpret_cast<const T *>(A.in) + job * A.in_stride;
  const T *lin = reinterpret_cast<const T *>(A.lam_in) + job * A.lam_stride;
  const T *table = reinterpret_cast<const T *>(A.table);
  T *out = reinterpret_cast<T *>(A.out) + job * A.out_stride;
  double *part = A.part + job * A.part_stride;
  const uint32_t gm = A.gate_mask;
  for (int i = 0; i <= ES; ++i) red[tid][i] = 0.0;

  if (A.kind == K_FWD || A.kind == K_WHT) {
    for (int x = tid; x < N; x += SMALL_NT) sp[x] = load_val<T>(A.load_mode, in, x, nmask, l0cs, n, A.em);
    __syncthreads();
    for (int b = 0; b < n; ++b) {
      if (!((gm >> b) & 1u)) continue;
      const T c = gcs[b].x, s = gcs[b].y;
      for (int pi = tid; pi < N / 2; pi += SMALL_NT) {
        const int x0 = ((pi >> b) << (b + 1)) | (pi & ((1 << b) - 1));
        const int x1 = x0 | (1 << b);
        const T a = sp[x0], bb = sp[x1];
        if (A.kind == K_WHT) {
          sp[x0] = a + bb;
          sp[x1] = a - bb;
        } else {
          sp[x0] = c * a - s * bb;
          sp[x1] = s * a + c * bb;
        }
      }
      __syncthreads();
    }
    if (cplx) {  // the pass's RZ gates as one phase per amplitude
      for (int x = 2 * tid; x < N; x += 2 * SMALL_NT) {
        const T2 ph = small_phase<T, T2>(x, gm, n, zcs);
        const T re = sp[x], im = sp[x + 1];
        sp[x] = re * ph.x - im * ph.y;
        sp[x + 1] = re * ph.y + im * ph.x;
      }
      __syncthreads();
    }
    for (int x = tid; x < N; x += SMALL_NT) {
      store_val(A.store_mode, out, x, nmask, sp[x], n, A.em);
      if (A.flags & F_ENERGY) red[tid][0] += (double)(sp[x] * sp[x] * table[x]);
    }
  } else if (A.kind == K_BWD) {
    const bool init = (A.flags & F_LAMBDA_INIT) != 0;
    for (int x = tid; x < N; x += SMALL_NT) {
      sp[x] = in[x];
      sl[x] = init ? table[x] * sp[x] : lin[x];
      if (A.flags & F_ENERGY) red[tid][ES] += (double)(sp[x] * sl[x]);
    }
    __syncthreads();
    for (int b = 0; b < n; ++b) {
      if (!((gm >> b) & 1u)) continue;
      for (int pi = tid; pi < N / 2; pi += SMALL_NT) {
        const int x0 = ((pi >> b) << (b + 1)) | (pi & ((1 << b) - 1));
        const int x1 = x0 | (1 << b);
        T g = sl[x1] * sp[x0] - sl[x0] * sp[x1];
        if (cplx) {  // cos(tz) Im<lam|Y|psi> - sin(tz) Im<lam|X|psi>, over amplitude pairs
          g *= zcs[b].x * zcs[b].x - zcs[b].y * zcs[b].y;
          if (!(x0 & 1)) {
            const T gx = sl[x0] * sp[x1 + 1] - sl[x0 + 1] * sp[x1] + sl[x1] * sp[x0 + 1] - sl[x1 + 1] * sp[x0];
            g -= 2 * zcs[b].x * zcs[b].y * gx;
          }
        }
        red[tid][b] += (double)g;
      }
    }
    if (cplx) {  // RZ gradients: sum_x s_q(x) Im(conj(lam) psi)
      for (int x = 2 * tid; x < N; x += 2 * SMALL_NT) {
        const T w = sl[x] * sp[x + 1] - sl[x + 1] * sp[x];
        for (int b = 1; b < n; ++b)
          if ((gm >> b) & 1u) red[tid][SMALL_MAXN + b] += (double)(((x >> b) & 1) ? -w : w);
      }
    }
    __syncthreads();
    if (cplx) {  // RZ(-theta) on lambda before the RY(-theta) rotations
      for (int x = 2 * tid; x < N; x += 2 * SMALL_NT) {
        const T2 ph = small_phase<T, T2>(x, gm, n, zcs);
        const T re = sl[x], im = sl[x + 1];
        sl[x] = re * ph.x + im * ph.y;
        sl[x + 1] = im * ph.x - re * ph.y;
      }
      __syncthreads();
    }
    for (int b = 0; b < n; ++b) {
      if (!((gm >> b) & 1u)) continue;
      const T c = gcs[b].x, s = -gcs[b].y;
      for (int pi = tid; pi < N / 2; pi += SMALL_NT) {
        const int x0 = ((pi >> b) << (b + 1)) | (pi & ((1 << b) - 1));
        const int x1 = x0 | (1 << b);
        const T a = sl[x0], bb = sl[x1];
        sl[x0] = c * a - s * bb;
        sl[x1] = s * a + c * bb;
      }
      __syncthreads();
    }
    for (int x = tid; x < N; x += SMALL_NT) store_val(A.store_mode, out, x, nmask, sl[x], n, A.em);
  } else if (A.kind == K_GRAD_L0) {
    const bool init = (A.flags & F_LAMBDA_INIT) != 0;
    for (int x = tid; x < N; x += SMALL_NT) {
      const T psi0 = product_state<T>(x, l0cs, n);
      const T lam = init ? table[x] * psi0 : lin[x];
      if (init) red[tid][ES] += (double)(psi0 * lam);
      for (int q = 0; q < n; ++q) {
        T wq = T(1);
        for (int i = 0; i < n; ++i) {
          const int b = (x >> i) & 1;
          wq *= (i == q) ? (b ? l0cs[i].x : -l0cs[i].y) : (b ? l0cs[i].y : l0cs[i].x);
        }
        red[tid][q] += (double)(lam * wq);
      }
    }
  } else if (A.kind == K_LAMBDA_XY) {
    for (int x = tid; x < N; x += SMALL_NT) {
      const T p = in[x];
      T acc = (A.flags & F_ACCUM) ? lin[x] : table[x] * p;
      for (int g = 0; g < A.ngroups; ++g) {
        const uint32_t u = (uint32_t)x ^ A.gmask[g];
        const T pu = in[u];
        T d = T(0);
        for (int j = A.gstart[g]; j < A.gstart[g + 1]; ++j)
          d += (__popc(u & A.tz[j]) & 1) ? -reinterpret_cast<const T *>(A.tc)[j]
                                           : reinterpret_cast<const T *>(A.tc)[j];
        acc += d * pu;
      }
      if (A.flags & F_WRITE_LAMBDA) out[x] = acc;
      red[tid][ES] += (double)(p * acc);
    }
  }
  __syncthreads();
  if (tid <= ES) {
    double s = 0.0;
    for (int i = 0; i < SMALL_NT; ++i) s += red[i][tid];
    const int q = tid;
    if (q < SMALL_MAXN) {
      const bool want = (A.kind == K_BWD && ((gm >> q) & 1u)) || (A.kind == K_GRAD_L0 && q < n);
      if (want) part[(long long)q * A.tiles] = s;
    } else if (q < ES && cplx && A.kind == K_BWD) {
      const int b = q - SMALL_MAXN;  // RZ rows follow the tb RY rows
      if ((gm >> b) & 1u) part[(long long)(A.tb + b) * A.tiles] = s;
    }
    if (A.kind == K_FWD && (A.flags & F_ENERGY) && q == 0) A.epart[job * A.part_stride] = s;
    if (q == ES && (A.flags & F_ENERGY) && A.kind != K_FWD) A.epart[job * A.part_stride] = s;
  }
}

// --------------------------------------------------------- small kernels --
template <typename T2>
__global__ void k_trig(const double *__restrict__ params, long long count, T2 *__restrict__ cs) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= count) return;
  double s, c;
  sincos(0.5 * params[i], &s, &c);
  T2 v;
  v.x = c;
  v.y = s;
  cs[i] = v;
}

__global__ void k_minlayer(const uint8_t *__restrict__ mask, int jobs, int n, int P, int none_value,
                           int *__restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= jobs) return;
  int m = none_value;
  if (mask == nullptr) {
    m = 0;
  } else {
    for (int p = 0; p < P; ++p)
      if (mask[(size_t)j * P + p]) {
        m = p / n;
        break;
      }
  }
  out[j] = m;
}

// One warp per output: lane-strided sum then an xor-shuffle tree (fixed order).
__global__ void k_reduce(const double *__restrict__ part, long long part_stride, const RedEntry *__restrict__ dir,
                         int ndir, const uint8_t *__restrict__ mask, int P, double *__restrict__ E,
                         double *__restrict__ grad) {
  const int wpb = blockDim.x / 32;
  const int e = blockIdx.x * wpb + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int job = blockIdx.y;
  if (e >= ndir) return;
  const RedEntry d = dir[e];
  const double *p = part + job * part_stride + d.off;
  double s = 0.0;
  for (int i = lane; i < d.count; i += 32) s += p[i];
  s = warp_sum(s);
  if (lane == 0) {
    if (d.param < 0) {
      E[job] = s;
    } else {
      const bool on = mask == nullptr || mask[(size_t)job * P + d.param] != 0;
      grad[(size_t)job * P + d.param] = on ? s : 0.0;
    }
  }
}

__global__ void k_scatter_coeffs(const uint32_t *__restrict__ z, const double *__restrict__ c, int count,
                                 double *__restrict__ table) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) table[z[i]] = c[i];
}

__global__ void k_convert_table(const double *__restrict__ src, float *__restrict__ dst, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

// The complex path's table: dst[2x + c] = src[x] (c = re/im channel), in the amplitude precision.
template <typename TD>
__global__ void k_expand_table(const double *__restrict__ src, TD *__restrict__ dst, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const TD v = (TD)src[i];
    dst[2 * i] = v;
    dst[2 * i + 1] = v;
  }
}

// Shifted parameter sets for Eq. 13: per job, row 0 = theta, then for each active
// parameter a (+pi/2, -pi/2) pair.
__global__ void k_shift_params(const double *__restrict__ params, int P, int jobs, const int *__restrict__ active,
                               int n_active, double *__restrict__ out) {
  const int rows = 2 * n_active + 1;
  const long long total = (long long)jobs * rows * P;
  const double half_pi = 1.5707963267948966;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(i % P);
    const long long r = (i / P) % rows;
    const long long j = i / ((long long)P * rows);
    double v = params[j * P + p];
    if (r > 0) {
      const int a = (int)((r - 1) / 2);
      if (active[a] == p) v += ((r - 1) % 2 == 0) ? half_pi : -half_pi;
    }
    out[i] = v;
  }
}

__global__ void k_shift_combine(const double *__restrict__ Es, int P, int jobs, const int *__restrict__ active,
                                int n_active, double *__restrict__ E, double *__restrict__ grad) {
  const int rows = 2 * n_active + 1;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)jobs * P) return;
  const int p = (int)(i % P);
  const long long j = i / P;
  const double *e = Es + j * rows;
  if (p == 0) E[j] = e[0];
  double g = 0.0;
  for (int a = 0; a < n_active; ++a)
    if (active[a] == p) g = 0.5 * (e[1 + 2 * a] - e[2 + 2 * a]);
  grad[i] = g;
}

}  // namespace

// --------------------------------------------------------------- launchers --
// The backward pass holds two tiles in shared memory (psi and lambda), and three
// CTAs share an SM: 2^13 FP32 or 2^12 FP64 amplitudes (64 KiB per CTA).
int max_tile_bits(int prec) { return prec ? 12 : 13; }

size_t pass_smem_bytes(int prec, int kind, int tb) {
  const size_t es = prec ? 8 : 4;
  if (tb < 10) return 0;
  if (kind == K_BWD) return 2 * (es << tb);
  if (kind == K_FWD || kind == K_WHT) return es << tb;
  return 0;
}

size_t xy_smem_bytes(int prec, int ngroups, int nterm) { return xy_layout(ngroups, nterm, prec ? 8 : 4).buf; }

template <typename T>
static cudaError_t launch_typed(const PassArgs &A, int jobs, int nterm, cudaStream_t s) {
  if (A.n <= SMALL_MAXN) {
    const dim3 grid(1, (unsigned)jobs);
    k_small<T><<<grid, SMALL_NT, 0, s>>>(A);
    return cudaGetLastError();
  }
  switch (A.tb) {
    case 10: return launch_tb<T, 10>(A, jobs, nterm, s);
    case 11: return launch_tb<T, 11>(A, jobs, nterm, s);
    case 12: return launch_tb<T, 12>(A, jobs, nterm, s);
    case 13:
      if constexpr (sizeof(T) == 4) return launch_tb<T, 13>(A, jobs, nterm, s);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

int num_sms_cached() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    n = (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0) ? v : 1;
  }
  return n;
}

// lambda = H psi for the X-mask groups on the complex path (amplitude y at
// u[2y], u[2y + 1]; A.n counts the index bits, n + 1).  Group g flips mask
// gmask[g]; each of its terms adds (tr + i ti) (-1)^popcount(u & tz) psi(u),
// u = y ^ gmask[g], with i^#Y folded into (tr, ti).  The diagonal part comes
// from the plain table E(y) (or lambda already written, F_ACCUM).  One CTA per
// XYC_PER_CTA amplitudes; the energy partial Re sum conj(psi) lambda per CTA.
constexpr int XYC_NT = 256;
constexpr int XYC_PER_CTA = XYC_AMPS_PER_CTA;

size_t xyc_smem_bytes(int prec, int ngroups, int nterm) {
  const size_t es = prec ? 8 : 4;
  auto up = [](size_t b) { return (b + 15) / 16 * 16; };
  return up((size_t)ngroups * 4) + up((size_t)(ngroups + 1) * 4) + up((size_t)nterm * 4) + 2 * up((size_t)nterm * es);
}

template <typename T>
__global__ void __launch_bounds__(XYC_NT) k_lambda_xy_c(const PassArgs A) {
  using T2 = typename V2<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double ered[XYC_NT / 32];
  const int ng = A.ngroups;
  const int t0 = ng > 0 ? A.gstart[0] : 0;
  const int nterm = ng > 0 ? A.gstart[ng] - t0 : 0;
  auto up = [](size_t b) { return (b + 15) / 16 * 16; };
  uint32_t *sgm = reinterpret_cast<uint32_t *>(smem_raw);
  int *sgs = reinterpret_cast<int *>(smem_raw + up((size_t)ng * 4));
  uint32_t *stz = reinterpret_cast<uint32_t *>(smem_raw + up((size_t)ng * 4) + up((size_t)(ng + 1) * 4));
  T *str = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(stz) + up((size_t)nterm * 4));
  T *sti = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(str) + up((size_t)nterm * sizeof(T)));
  const int tid = threadIdx.x;
  for (int i = tid; i < ng; i += XYC_NT) sgm[i] = A.gmask[i];
  for (int i = tid; i <= ng; i += XYC_NT) sgs[i] = A.gstart[i] - t0;
  for (int i = tid; i < nterm; i += XYC_NT) {
    stz[i] = A.tz[t0 + i];
    str[i] = reinterpret_cast<const T *>(A.tc)[t0 + i];
    sti[i] = reinterpret_cast<const T *>(A.tci)[t0 + i];
  }
  __syncthreads();
  const int job = blockIdx.y;
  const long long NQ = 1LL << (A.n - 1);
  const T2 *in = reinterpret_cast<const T2 *>(A.in) + (size_t)job * (A.in_stride / 2);
  const T2 *lin = reinterpret_cast<const T2 *>(A.lam_in) + (size_t)job * (A.lam_stride / 2);
  T2 *out = reinterpret_cast<T2 *>(A.out) + (size_t)job * (A.out_stride / 2);
  const T *table = reinterpret_cast<const T *>(A.table);
  T eacc = T(0);
  for (int k = 0; k < XYC_PER_CTA / XYC_NT; ++k) {
    const long long y = (long long)blockIdx.x * XYC_PER_CTA + k * XYC_NT + tid;
    if (y >= NQ) break;
    const T2 p = __ldcg(in + y);
    T2 acc;
    if (A.flags & F_ACCUM) {
      acc = lin[y];
    } else {
      const T e = table[y];
      acc.x = e * p.x;
      acc.y = e * p.y;
    }
    for (int g = 0; g < ng; ++g) {
      const uint32_t u = (uint32_t)y ^ sgm[g];
      const T2 pu = __ldcg(in + u);
      T dr = T(0), di = T(0);
      for (int j = sgs[g]; j < sgs[g + 1]; ++j) {
        const bool neg = __popc(u & stz[j]) & 1;
        dr += neg ? -str[j] : str[j];
        di += neg ? -sti[j] : sti[j];
      }
      acc.x += dr * pu.x - di * pu.y;
      acc.y += dr * pu.y + di * pu.x;
    }
    if (A.flags & F_WRITE_LAMBDA) out[y] = acc;
    eacc += p.x * acc.x + p.y * acc.y;
  }
  if (A.flags & F_ENERGY) {
    for (int o = 16; o > 0; o >>= 1) eacc += __shfl_xor_sync(0xffffffffu, eacc, o);
    if ((tid & 31) == 0) ered[tid >> 5] = (double)eacc;
    __syncthreads();
    if (tid == 0) {
      double e = 0.0;
      for (int w = 0; w < XYC_NT / 32; ++w) e += ered[w];
      A.epart[(size_t)job * A.part_stride + blockIdx.x] = e;
    }
  }
}

cudaError_t launch_pass(int prec, const PassArgs &A, int jobs, int nterm, cudaStream_t s) {
  if (jobs < 1 || A.tiles < 1) return cudaErrorInvalidValue;
  if (A.kind >= K_MPS) return launch_mps(prec, A, jobs, s);
  if (A.kind == K_LAMBDA_XY && (A.flags & F_COMPLEX)) {
    const size_t smem = xyc_smem_bytes(prec, A.ngroups, nterm);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)A.tiles, (unsigned)jobs);
    if (prec) {
      if (smem > 48 * 1024) cudaFuncSetAttribute(k_lambda_xy_c<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_lambda_xy_c<double><<<grid, XYC_NT, smem, s>>>(A);
    } else {
      if (smem > 48 * 1024) cudaFuncSetAttribute(k_lambda_xy_c<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_lambda_xy_c<float><<<grid, XYC_NT, smem, s>>>(A);
    }
    return cudaGetLastError();
  }
  if (A.kind == K_GRAD_L0 && A.n > SMALL_MAXN) return launch_grad_l0(prec, A, jobs, s);
  return prec ? launch_typed<double>(A, jobs, nterm, s) : launch_typed<float>(A, jobs, nterm, s);
}

cudaError_t launch_trig(int prec, const double *params, long long count, void *cs, cudaStream_t s) {
  const int bs = 256;
  const unsigned gs = (unsigned)((count + bs - 1) / bs);
  if (count <= 0) return cudaSuccess;
  if (prec)
    k_trig<double2><<<gs, bs, 0, s>>>(params, count, reinterpret_cast<double2 *>(cs));
  else
    k_trig<float2><<<gs, bs, 0, s>>>(params, count, reinterpret_cast<float2 *>(cs));
  return cudaGetLastError();
}

cudaError_t launch_minlayer(const uint8_t *mask, int jobs, int n, int P, int none_value, int *out,
                            cudaStream_t s) {
  k_minlayer<<<(jobs + 127) / 128, 128, 0, s>>>(mask, jobs, n, P, none_value, out);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const double *part, long long part_stride, const RedEntry *dir, int ndir,
                          const uint8_t *mask, int P, double *E, double *grad, int jobs, cudaStream_t s) {
  if (ndir <= 0) return cudaSuccess;
  const int wpb = 8;
  const dim3 grid((unsigned)((ndir + wpb - 1) / wpb), (unsigned)jobs);
  k_reduce<<<grid, wpb * 32, 0, s>>>(part, part_stride, dir, ndir, mask, P, E, grad);
  return cudaGetLastError();
}

cudaError_t launch_scatter_coeffs(const uint32_t *z, const double *c, int count, double *table,
                                  cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_scatter_coeffs<<<(count + 255) / 256, 256, 0, s>>>(z, c, count, table);
  return cudaGetLastError();
}

cudaError_t launch_convert_table(const double *src, float *dst, long long count, cudaStream_t s) {
  const long long blocks = (count + 255) / 256;
  k_convert_table<<<(unsigned)(blocks < 65536 ? blocks : 65536), 256, 0, s>>>(src, dst, count);
  return cudaGetLastError();
}

cudaError_t launch_expand_table(const double *src, void *dst, long long count, int prec, cudaStream_t s) {
  const long long blocks = (count + 255) / 256;
  const unsigned g = (unsigned)(blocks < 65536 ? blocks : 65536);
  if (prec)
    k_expand_table<double><<<g, 256, 0, s>>>(src, (double *)dst, count);
  else
    k_expand_table<float><<<g, 256, 0, s>>>(src, (float *)dst, count);
  return cudaGetLastError();
}

cudaError_t launch_shift_params(const double *params, int P, int jobs, const int *active, int n_active,
                                double *out, cudaStream_t s) {
  const long long total = (long long)jobs * (2 * n_active + 1) * P;
  const long long blocks = (total + 255) / 256;
  k_shift_params<<<(unsigned)(blocks < 65536 ? blocks : 65536), 256, 0, s>>>(params, P, jobs, active, n_active, out);
  return cudaGetLastError();
}

cudaError_t launch_shift_combine(const double *Es, int P, int jobs, const int *active, int n_active, double *E,
                                 double *grad, cudaStream_t s) {
  const long long total = (long long)jobs * P;
  k_shift_combine<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(Es, P, jobs, active, n_active, E, grad);
  return cudaGetLastError();
}

}  // namespace gvqe
