// gvqe_kernels.cu -- sm_103a kernels of the Graph-VQE energy / gradient engine.
//
// The tile engine (tile bits tb >= 10): a CTA owns one tile of 2^tb real
// amplitudes; each of its 2^(tb-5) threads holds 32 amplitudes in registers
// at a time, and the tile moves through three register "rounds":
//   round L: registers <-> tile bits 5..9, lanes <-> bits 0..4, warps <-> bits 10..
//            (global loads/stores here are coalesced 128-byte warp accesses)
//   round M: registers <-> tile bits 0..4 (one 32-amplitude group per thread,
//            16-byte vector shared-memory accesses)
//   round H: registers <-> tile bits 10..tb-1
// RY gates on the bits held in registers are applied in registers; shared
// memory is only the transpose between rounds.  The shared-memory tile is
// swizzled (16-byte chunk index XOR group index) so both access shapes are
// free of bank conflicts.
//
// Registers smaller than 2^10 amplitudes use a plain whole-state kernel
// (k_small) with one butterfly sweep per bit.
//
// Accumulation: energies and gradients sum one thread's products and one
// warp's lanes in the amplitude precision, then everything above a warp in
// FP64 in a fixed order (deterministic).
#include <cstdio>

#include "gvqe_engine.cuh"

namespace gvqe {

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

constexpr int ROUND = 32;  // amplitudes per thread per round (5 register bits)

// ----------------------------------------------------------------- helpers --

template <typename T>
__device__ __forceinline__ int swz(int i) {
  constexpr int CH = 16 / (int)sizeof(T);  // amplitudes per 16-byte chunk
  return i ^ (((i >> 5) & 7) * CH);
}

__device__ __forceinline__ long long tile_of_block(long long bx, long long tiles, bool pair) {
  if (!pair || tiles < 2) return bx;
  const long long u = bx >> 1;
  return (bx & 1) ? (u ^ (tiles - 1)) : u;
}

__device__ __forceinline__ long long tile_base(long long t, int c, int a, int tb) {
  const int lo = a - c;
  const long long tlo = t & ((1LL << lo) - 1);
  const long long thi = t >> lo;
  return (tlo << c) | (thi << (a + tb - c));
}

struct Layout {
  long long tbase;
  int c, a;
  int cmask;
  __device__ __forceinline__ long long g(int i) const {
    return tbase | (long long)(i & cmask) | ((long long)(i >> c) << a);
  }
};

// x = A^-1 y for the linear CX chain (y = prefix XOR of x).
__device__ __forceinline__ long long cx_inv(long long y, long long nmask) {
  return (y ^ (y << 1)) & nmask;
}

template <typename T, typename T2>
__device__ __forceinline__ T product_state(long long x, const T2 *l0, int n) {
  T p = T(1);
  for (int q = 0; q < n; ++q) p *= ((x >> q) & 1) ? l0[q].y : l0[q].x;
  return p;
}

template <typename T, typename T2>
__device__ __forceinline__ T load_val(int mode, const T *__restrict__ in, long long y, long long nmask,
                                      const T2 *l0, int n) {
  switch (mode) {
    case LD_GATHER:
      return in[cx_inv(y, nmask)];
    case LD_L0_GATHER:
      return product_state<T>(cx_inv(y, nmask), l0, n);
    case LD_L0:
      return product_state<T>(y, l0, n);
    default:
      return in[y];
  }
}

template <typename T>
__device__ __forceinline__ void store_val(int mode, T *__restrict__ out, long long y, long long nmask, T v) {
  if (mode == ST_PLAIN)
    out[y] = v;
  else if (mode == ST_SCATTER)
    out[cx_inv(y, nmask)] = v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// RY on register bit JB: (a, b) -> (c a - s b, s a + c b).
template <int JB, typename T>
__device__ __forceinline__ void rot_bit(T (&v)[ROUND], T c, T s) {
#pragma unroll
  for (int k = 0; k < ROUND; ++k) {
    if (k & (1 << JB)) continue;
    const T a = v[k], b = v[k | (1 << JB)];
    v[k] = c * a - s * b;
    v[k | (1 << JB)] = s * a + c * b;
  }
}

// Unnormalised Walsh-Hadamard butterfly on register bit JB: (a, b) -> (a + b, a - b).
template <int JB, typename T>
__device__ __forceinline__ void wht_bit(T (&v)[ROUND]) {
#pragma unroll
  for (int k = 0; k < ROUND; ++k) {
    if (k & (1 << JB)) continue;
    const T a = v[k], b = v[k | (1 << JB)];
    v[k] = a + b;
    v[k | (1 << JB)] = a - b;
  }
}

// Im<lam|Y_q|psi> restricted to this thread's pairs along register bit JB:
// sum over pairs (x0, x1 = x0 | bit) of lam[x1] psi[x0] - lam[x0] psi[x1].
template <int JB, typename T>
__device__ __forceinline__ T grad_bit(const T (&psi)[ROUND], const T (&lam)[ROUND]) {
  T acc = T(0);
#pragma unroll
  for (int k = 0; k < ROUND; ++k) {
    if (k & (1 << JB)) continue;
    acc += lam[k | (1 << JB)] * psi[k] - lam[k] * psi[k | (1 << JB)];
  }
  return acc;
}

// Gates of one round: register bit j (< NB) holds tile bit tbit0 + j.
template <int NB, bool WHT, typename T, typename T2>
__device__ __forceinline__ void round_gates(T (&v)[ROUND], const T2 *gcs, uint32_t gmask, int tbit0,
                                            bool inverse) {
#define GVQE_GATE(J)                                             \
  if (NB > J && ((gmask >> (tbit0 + J)) & 1u)) {                 \
    if (WHT) {                                                   \
      wht_bit<J>(v);                                             \
    } else {                                                     \
      const T2 cs = gcs[tbit0 + J];                              \
      rot_bit<J>(v, cs.x, inverse ? -cs.y : cs.y);               \
    }                                                            \
  }
  GVQE_GATE(0)
  GVQE_GATE(1)
  GVQE_GATE(2)
  GVQE_GATE(3)
  GVQE_GATE(4)
#undef GVQE_GATE
}

// Gradient partials of one round, reduced over the warp; lane 0 stores them.
template <int NB, typename T>
__device__ __forceinline__ void round_grads(const T (&psi)[ROUND], const T (&lam)[ROUND], uint32_t gmask,
                                            int tbit0, double *wred /* [16] of this warp */, int lane) {
#define GVQE_GRAD(J)                                      \
  if (NB > J && ((gmask >> (tbit0 + J)) & 1u)) {          \
    const T gsum = warp_sum(grad_bit<J>(psi, lam));       \
    if (lane == 0) wred[tbit0 + J] = (double)gsum;        \
  }
  GVQE_GRAD(0)
  GVQE_GRAD(1)
  GVQE_GRAD(2)
  GVQE_GRAD(3)
  GVQE_GRAD(4)
#undef GVQE_GRAD
}

// ------------------------------------------------ round index arithmetic --
// Round L: element k of thread (lane, warp w) is tile index lane | k<<5 | w<<10.
__device__ __forceinline__ int idx_L(int lane, int w, int k) { return lane | (k << 5) | (w << 10); }
// Round H: thread tid handles groups tid + it*NT; element k = it<<H | j is index group | j<<10.
template <int TB>
__device__ __forceinline__ int idx_H(int tid, int k) {
  constexpr int H = TB - 10;
  constexpr int NT = 1 << (TB - 5);
  const int it = k >> H, j = k & ((1 << H) - 1);
  return (tid + it * NT) | (j << 10);
}

template <typename T>
__device__ __forceinline__ void lds_M(const T *s, int G, T (&v)[ROUND]) {
  // 32 consecutive amplitudes of group G as 16-byte chunks (swizzled chunk order).
  constexpr int CH = 16 / (int)sizeof(T);
  using T2 = typename V2<T>::type;
#pragma unroll
  for (int c = 0; c < ROUND / CH; ++c) {
    const int pc = c ^ (G & 7);
    if constexpr (CH == 4) {
      const float4 q = *reinterpret_cast<const float4 *>(s + (G << 5) + pc * 4);
      v[4 * c + 0] = q.x;
      v[4 * c + 1] = q.y;
      v[4 * c + 2] = q.z;
      v[4 * c + 3] = q.w;
    } else {
      const T2 q = *reinterpret_cast<const T2 *>(s + (G << 5) + pc * 2);
      v[2 * c + 0] = q.x;
      v[2 * c + 1] = q.y;
    }
  }
}

template <typename T>
__device__ __forceinline__ void sts_M(T *s, int G, const T (&v)[ROUND]) {
  constexpr int CH = 16 / (int)sizeof(T);
  using T2 = typename V2<T>::type;
#pragma unroll
  for (int c = 0; c < ROUND / CH; ++c) {
    const int pc = c ^ (G & 7);
    if constexpr (CH == 4) {
      *reinterpret_cast<float4 *>(s + (G << 5) + pc * 4) =
          make_float4(v[4 * c + 0], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
    } else {
      T2 q;
      q.x = v[2 * c + 0];
      q.y = v[2 * c + 1];
      *reinterpret_cast<T2 *>(s + (G << 5) + pc * 2) = q;
    }
  }
}

template <int TB, typename T>
__device__ __forceinline__ void lds_H(const T *s, int tid, T (&v)[ROUND]) {
#pragma unroll
  for (int k = 0; k < ROUND; ++k) v[k] = s[swz<T>(idx_H<TB>(tid, k))];
}
template <int TB, typename T>
__device__ __forceinline__ void sts_H(T *s, int tid, const T (&v)[ROUND]) {
#pragma unroll
  for (int k = 0; k < ROUND; ++k) s[swz<T>(idx_H<TB>(tid, k))] = v[k];
}
template <typename T>
__device__ __forceinline__ void lds_L(const T *s, int lane, int w, T (&v)[ROUND]) {
#pragma unroll
  for (int k = 0; k < ROUND; ++k) v[k] = s[swz<T>(idx_L(lane, w, k))];
}
template <typename T>
__device__ __forceinline__ void sts_L(T *s, int lane, int w, const T (&v)[ROUND]) {
#pragma unroll
  for (int k = 0; k < ROUND; ++k) s[swz<T>(idx_L(lane, w, k))] = v[k];
}

// Sum NW per-warp doubles in warp order (deterministic), returns the total.
template <int NW>
__device__ __forceinline__ double sum_warps(const double *x) {
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < NW; ++w) s += x[w];
  return s;
}

// Shared prologue: per-tile-bit gate coefficients and layer-0 coefficients.
template <typename T2>
__device__ __forceinline__ void load_coeffs(const PassArgs &A, const T2 *cs, T2 *gcs, T2 *l0cs, int tid) {
  if (tid < 16) {
    T2 v;
    v.x = 1;
    v.y = 0;
    if (tid < A.tb && ((A.gate_mask >> tid) & 1u) && A.kind != K_WHT) {
      const int q = tid < A.c ? tid : A.a + tid - A.c;
      v = cs[A.layer * A.n + q];
    }
    gcs[tid] = v;
  }
  if (tid < 32 && tid < A.n && l0cs != nullptr &&
      (A.load_mode == LD_L0 || A.load_mode == LD_L0_GATHER || A.kind == K_GRAD_L0))
    l0cs[tid] = cs[tid];
}

// ------------------------------------------------------ forward tile pass --
template <typename T, int TB, bool WHT>
__global__ void __launch_bounds__(1 << (TB - 5)) k_fwd(const PassArgs A) {
  using T2 = typename V2<T>::type;
  constexpr int NT = 1 << (TB - 5);
  constexpr int NW = NT / 32;
  constexpr int H = TB - 10;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *s = reinterpret_cast<T *>(smem_raw);
  __shared__ T2 gcs[16];
  __shared__ T2 l0cs[32];
  __shared__ double ered[NW];

  const int job = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long t = tile_of_block(blockIdx.x, A.tiles, (A.flags & F_PAIR_ORDER) != 0);
  const Layout L{tile_base(t, A.c, A.a, TB), A.c, A.a, (1 << A.c) - 1};
  const long long nmask = (1LL << A.n) - 1;
  const T2 *cs = reinterpret_cast<const T2 *>(A.cs) + (size_t)(A.job0 + job) * A.P;
  if (!WHT) load_coeffs(A, cs, gcs, l0cs, tid);
  __syncthreads();
  const T *in = reinterpret_cast<const T *>(A.in) + job * A.in_stride;
  T *out = reinterpret_cast<T *>(A.out) + job * A.out_stride;
  const uint32_t gm = A.gate_mask;

  T v[ROUND];
  // round L: global -> registers (tile bits 5..9) -> gates -> shared
#pragma unroll
  for (int k = 0; k < ROUND; ++k) v[k] = load_val<T>(A.load_mode, in, L.g(idx_L(lane, w, k)), nmask, l0cs, A.n);
  round_gates<5, WHT>(v, gcs, gm, 5, false);
  sts_L(s, lane, w, v);
  __syncthreads();
  // round M: tile bits 0..4
  if (gm & 0x1Fu) {
    lds_M(s, tid, v);
    round_gates<5, WHT>(v, gcs, gm, 0, false);
    sts_M(s, tid, v);
    __syncthreads();
  }
  // round H: tile bits 10..tb-1, then the store and the energy epilogue
  lds_H<TB>(s, tid, v);
  round_gates<H, WHT>(v, gcs, gm, 10, false);
  T eacc = T(0);
  const T *table = reinterpret_cast<const T *>(A.table);
#pragma unroll
  for (int k = 0; k < ROUND; ++k) {
    const long long y = L.g(idx_H<TB>(tid, k));
    store_val(A.store_mode, out, y, nmask, v[k]);
    if (A.flags & F_ENERGY) eacc += v[k] * v[k] * table[y];
  }
  if (A.flags & F_ENERGY) {
    eacc = warp_sum(eacc);
    if (lane == 0) ered[w] = (double)eacc;
    __syncthreads();
    if (tid == 0) A.epart[job * A.part_stride + t] = sum_warps<NW>(ered);
  }
}

// ------------------------------------------------------ backward tile pass --
// lambda and psi are both at the point right after this pass's gates.  Rounds
// L, M, H read both and form the gradients (all at that same point); round H
// then applies RY(-theta) to lambda on its bits, rounds M and L follow on
// theirs, and round L writes lambda (through the inverse CX chain for the
// first pass of a layer).
template <typename T, int TB>
__global__ void __launch_bounds__(1 << (TB - 5)) k_bwd(const PassArgs A) {
  using T2 = typename V2<T>::type;
  constexpr int NT = 1 << (TB - 5);
  constexpr int NW = NT / 32;
  constexpr int H = TB - 10;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sp = reinterpret_cast<T *>(smem_raw);
  T *sl = sp + (1 << TB);
  __shared__ T2 gcs[16];
  __shared__ double gred[NW][16];
  __shared__ double ered[NW];

  const int job = blockIdx.y;
  if (A.minlayer != nullptr && !(A.flags & F_ENERGY) && A.layer < A.minlayer[A.job0 + job]) return;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long t = tile_of_block(blockIdx.x, A.tiles, (A.flags & F_PAIR_ORDER) != 0);
  const Layout L{tile_base(t, A.c, A.a, TB), A.c, A.a, (1 << A.c) - 1};
  const long long nmask = (1LL << A.n) - 1;
  const T2 *cs = reinterpret_cast<const T2 *>(A.cs) + (size_t)(A.job0 + job) * A.P;
  load_coeffs<T2>(A, cs, gcs, nullptr, tid);
  __syncthreads();
  const T *in = reinterpret_cast<const T *>(A.in) + job * A.in_stride;
  const T *lin = reinterpret_cast<const T *>(A.lam_in) + job * A.lam_stride;
  const T *table = reinterpret_cast<const T *>(A.table);
  T *out = reinterpret_cast<T *>(A.out) + job * A.out_stride;
  const uint32_t gm = A.gate_mask;
  const bool init = (A.flags & F_LAMBDA_INIT) != 0;

  T psi[ROUND], lam[ROUND];
  T eacc = T(0);
  // round L
#pragma unroll
  for (int k = 0; k < ROUND; ++k) {
    const long long y = L.g(idx_L(lane, w, k));
    psi[k] = in[y];
    lam[k] = init ? table[y] * psi[k] : lin[y];
    eacc += psi[k] * lam[k];
  }
  round_grads<5>(psi, lam, gm, 5, gred[w], lane);
  sts_L(sp, lane, w, psi);
  sts_L(sl, lane, w, lam);
  if (A.flags & F_ENERGY) {
    eacc = warp_sum(eacc);
    if (lane == 0) ered[w] = (double)eacc;
  }
  __syncthreads();
  // round M (gradients only)
  if (gm & 0x1Fu) {
    lds_M(sp, tid, psi);
    lds_M(sl, tid, lam);
    round_grads<5>(psi, lam, gm, 0, gred[w], lane);
  }
  // round H: gradients, then RY(-theta) on lambda
  lds_H<TB>(sp, tid, psi);
  lds_H<TB>(sl, tid, lam);
  round_grads<H>(psi, lam, gm, 10, gred[w], lane);
  round_gates<H, false>(lam, gcs, gm, 10, true);
  __syncthreads();  // every thread has read the tile before lambda is overwritten
  sts_H<TB>(sl, tid, lam);
  __syncthreads();
  if (gm & 0x1Fu) {
    lds_M(sl, tid, lam);
    round_gates<5, false>(lam, gcs, gm, 0, true);
    sts_M(sl, tid, lam);
    __syncthreads();
  }
  lds_L(sl, lane, w, lam);
  round_gates<5, false>(lam, gcs, gm, 5, true);
#pragma unroll
  for (int k = 0; k < ROUND; ++k) store_val(A.store_mode, out, L.g(idx_L(lane, w, k)), nmask, lam[k]);

  double *part = A.part + job * A.part_stride;
  if (tid < TB && ((gm >> tid) & 1u)) {
    double g = 0.0;
#pragma unroll
    for (int ww = 0; ww < NW; ++ww) g += gred[ww][tid];
    part[(long long)tid * A.tiles + t] = g;
  }
  if ((A.flags & F_ENERGY) && tid == 0) A.epart[job * A.part_stride + t] = sum_warps<NW>(ered);
}

// ------------------------------------------------ layer-0 gradient pass --
// g_{0,q} = sum_x lambda_0[x] prod_{q' != q} f_q'(x_q') d_q(x_q) with
// f(0) = cos(t/2), f(1) = sin(t/2), d(0) = -sin(t/2), d(1) = cos(t/2): the
// adjoint formula evaluated against the layer-0 product state.  The tile is
// global bits [0, tb); the product over the register bits 5..9 is tabulated.
template <typename T, int TB>
__global__ void __launch_bounds__(1 << (TB - 5)) k_grad_l0(const PassArgs A) {
  using T2 = typename V2<T>::type;
  constexpr int NT = 1 << (TB - 5);
  constexpr int NW = NT / 32;
  constexpr int NV = 11;  // per-thread values reduced over the warp
  __shared__ T2 l0cs[32];
  __shared__ T2 gcs_unused[16];
  __shared__ T RF[ROUND], RD[5][ROUND];
  __shared__ double wv[NW][NV];
  __shared__ double ered[NW];
  __shared__ double fhi_d[32];
  __shared__ double fhi_all;

  const int job = blockIdx.y;
  if (A.minlayer != nullptr && !(A.flags & F_ENERGY) && A.minlayer[A.job0 + job] > 0) return;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long t = blockIdx.x;
  const int n = A.n;
  const T2 *cs = reinterpret_cast<const T2 *>(A.cs) + (size_t)(A.job0 + job) * A.P;
  load_coeffs<T2>(A, cs, gcs_unused, l0cs, tid);
  __syncthreads();
  if (tid < ROUND) {
    // RF[k] = prod_j f_{5+j}(k_j); RD[j][k] replaces factor j by d.
    T f = T(1);
    for (int j = 0; j < 5; ++j) {
      const T2 c = l0cs[5 + j];
      f *= ((tid >> j) & 1) ? c.y : c.x;
    }
    RF[tid] = f;
    for (int j = 0; j < 5; ++j) {
      T g = T(1);
      for (int i = 0; i < 5; ++i) {
        const T2 c = l0cs[5 + i];
        const int b = (tid >> i) & 1;
        g *= (i == j) ? (b ? c.x : -c.y) : (b ? c.y : c.x);
      }
      RD[j][tid] = g;
    }
  }
  if (tid < 32) {
    // factors of the tile's own bits q >= TB
    const int q = TB + tid;
    if (tid == 0) {
      double f = 1.0;
      for (int qq = TB; qq < n; ++qq) {
        const T2 c = l0cs[qq];
        f *= ((t >> (qq - TB)) & 1) ? (double)c.y : (double)c.x;
      }
      fhi_all = f;
    }
    if (q < n) {
      double f = 1.0;
      for (int qq = TB; qq < n; ++qq) {
        const T2 c = l0cs[qq];
        const int b = (int)((t >> (qq - TB)) & 1);
        f *= (qq == q) ? (b ? (double)c.x : -(double)c.y) : (b ? (double)c.y : (double)c.x);
      }
      fhi_d[tid] = f;
    }
  }
  __syncthreads();

  // lane factors (tile bits 0..4) and their d-variants
  T lane_f = T(1), lane_d[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const T2 c = l0cs[j];
    lane_f *= ((lane >> j) & 1) ? c.y : c.x;
  }
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    T g = T(1);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const T2 c = l0cs[i];
      const int b = (lane >> i) & 1;
      g *= (i == j) ? (b ? c.x : -c.y) : (b ? c.y : c.x);
    }
    lane_d[j] = g;
  }
  T warp_f = T(1);
  for (int j = 10; j < TB; ++j) {
    const T2 c = l0cs[j];
    warp_f *= ((w >> (j - 10)) & 1) ? c.y : c.x;
  }

  const bool init = (A.flags & F_LAMBDA_INIT) != 0;
  const T *lin = reinterpret_cast<const T *>(A.lam_in) + job * A.lam_stride;
  const T *table = reinterpret_cast<const T *>(A.table);
  const long long tbase = t << TB;
  const T fhi_t = (T)fhi_all;
  T S = T(0), Sj[5] = {T(0), T(0), T(0), T(0), T(0)};
  T eacc = T(0);
#pragma unroll
  for (int k = 0; k < ROUND; ++k) {
    const long long x = tbase | idx_L(lane, w, k);
    T lam;
    if (init) {
      const T psi0 = lane_f * RF[k] * warp_f * fhi_t;
      lam = table[x] * psi0;
      eacc += psi0 * lam;
    } else {
      lam = lin[x];
    }
    S += lam * RF[k];
#pragma unroll
    for (int j = 0; j < 5; ++j) Sj[j] += lam * RD[j][k];
  }
  T vals[NV];
  vals[0] = lane_f * S;
#pragma unroll
  for (int j = 0; j < 5; ++j) vals[1 + j] = lane_f * Sj[j];
#pragma unroll
  for (int j = 0; j < 5; ++j) vals[6 + j] = lane_d[j] * S;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const T r = warp_sum(vals[i]);
    if (lane == 0) wv[w][i] = (double)r;
  }
  if (init) {
    eacc = warp_sum(eacc);
    if (lane == 0) ered[w] = (double)eacc;
  }
  __syncthreads();

  double *part = A.part + job * A.part_stride;
  if (tid < n) {
    const int q = tid;
    double g = 0.0;
    const double fh = fhi_all;
    for (int ww = 0; ww < NW; ++ww) {
      double wf = 1.0, wd = 1.0;
      for (int j = 10; j < TB; ++j) {
        const T2 c = l0cs[j];
        const int b = (ww >> (j - 10)) & 1;
        const double fj = b ? (double)c.y : (double)c.x;
        wf *= fj;
        wd *= (j == q) ? (b ? (double)c.x : -(double)c.y) : fj;
      }
      if (q < 5)
        g += wf * wv[ww][6 + q];
      else if (q < 10)
        g += wf * wv[ww][1 + (q - 5)];
      else if (q < TB)
        g += wd * wv[ww][0];
      else
        g += wf * wv[ww][0];
    }
    g *= (q < TB) ? fh : fhi_d[q - TB];
    part[(long long)q * A.tiles + t] = g;
  }
  if (init && tid == 0) A.epart[job * A.part_stride + t] = sum_warps<NW>(ered);
}

// Shared-memory layout of one chunk of X-mask groups: [gmask][gstart][tz][tc], 16-byte aligned parts.
struct XyLayout {
  size_t gm, gs, tz, tc, total;
};
__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline XyLayout xy_layout(int ngroups, int nterm, int elem) {
  XyLayout l;
  l.gm = 0;
  l.gs = align16((size_t)ngroups * 4);
  l.tz = align16(l.gs + (size_t)(ngroups + 1) * 4);
  l.tc = align16(l.tz + (size_t)nterm * 4);
  l.total = align16(l.tc + (size_t)nterm * elem);
  return l;
}

// ----------------------------------------- lambda = H psi with X-mask groups --
// lambda[x] = E(x) psi[x] + sum_groups D_m(x ^ m) psi[x ^ m] with
// D_m(u) = sum_{k in group} c_k (-1)^popcount(u & z_k) (c_k carries the i^#Y sign).
template <typename T, int TB>
__global__ void __launch_bounds__(1 << (TB - 5)) k_lambda_xy(const PassArgs A) {
  constexpr int NT = 1 << (TB - 5);
  constexpr int NW = NT / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nterm = A.ngroups > 0 ? A.gstart[A.ngroups] - A.gstart[0] : 0;
  const XyLayout lay = xy_layout(A.ngroups, nterm, (int)sizeof(T));
  uint32_t *sgm = reinterpret_cast<uint32_t *>(smem_raw + lay.gm);
  int *sgs = reinterpret_cast<int *>(smem_raw + lay.gs);
  uint32_t *stz = reinterpret_cast<uint32_t *>(smem_raw + lay.tz);
  T *stc = reinterpret_cast<T *>(smem_raw + lay.tc);
  __shared__ double ered[NW];
  const int job = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long t = blockIdx.x;
  const int t0 = A.ngroups > 0 ? A.gstart[0] : 0;
  for (int i = tid; i < A.ngroups; i += NT) sgm[i] = A.gmask[i];
  for (int i = tid; i <= A.ngroups; i += NT) sgs[i] = A.gstart[i] - t0;
  for (int i = tid; i < nterm; i += NT) {
    stz[i] = A.tz[t0 + i];
    stc[i] = reinterpret_cast<const T *>(A.tc)[t0 + i];
  }
  __syncthreads();
  const T *in = reinterpret_cast<const T *>(A.in) + job * A.in_stride;
  const T *lin = reinterpret_cast<const T *>(A.lam_in) + job * A.lam_stride;
  const T *table = reinterpret_cast<const T *>(A.table);
  T *out = reinterpret_cast<T *>(A.out) + job * A.out_stride;
  const long long tbase = t << TB;
  T eacc = T(0);
  for (int k = 0; k < ROUND; ++k) {
    const long long x = tbase | idx_L(lane, w, k);
    const T p = in[x];
    T acc = (A.flags & F_ACCUM) ? lin[x] : table[x] * p;
    for (int g = 0; g < A.ngroups; ++g) {
      const long long u = x ^ (long long)sgm[g];
      const T pu = in[u];
      T d = T(0);
      const uint32_t ul = (uint32_t)u;
      for (int j = sgs[g]; j < sgs[g + 1]; ++j) d += (__popc(ul & stz[j]) & 1) ? -stc[j] : stc[j];
      acc += d * pu;
    }
    if (A.flags & F_WRITE_LAMBDA) out[x] = acc;
    eacc += p * acc;
  }
  if (A.flags & F_ENERGY) {
    eacc = warp_sum(eacc);
    if (lane == 0) ered[w] = (double)eacc;
    __syncthreads();
    if (tid == 0) A.epart[job * A.part_stride + t] = sum_warps<NW>(ered);
  }
}

// --------------------------------------------- whole-register kernel (n < 10) --
// One CTA per job holds the whole state (2^n <= 512 amplitudes) and applies
// the pass one gate bit at a time.  Reductions are per-thread FP64 partials
// summed in thread order.
constexpr int SMALL_NT = 128;
constexpr int SMALL_MAXN = 9;

template <typename T>
__global__ void __launch_bounds__(SMALL_NT) k_small(const PassArgs A) {
  using T2 = typename V2<T>::type;
  __shared__ T sp[1 << SMALL_MAXN], sl[1 << SMALL_MAXN];
  __shared__ T2 gcs[16];
  __shared__ T2 l0cs[32];
  __shared__ double red[SMALL_NT][SMALL_MAXN + 1];
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
  if (A.kind != K_WHT) load_coeffs(A, cs, gcs, l0cs, tid);
  __syncthreads();
  const T *in = reinterpret_cast<const T *>(A.in) + job * A.in_stride;
  const T *lin = reinterpret_cast<const T *>(A.lam_in) + job * A.lam_stride;
  const T *table = reinterpret_cast<const T *>(A.table);
  T *out = reinterpret_cast<T *>(A.out) + job * A.out_stride;
  double *part = A.part + job * A.part_stride;
  const uint32_t gm = A.gate_mask;
  for (int i = 0; i <= SMALL_MAXN; ++i) red[tid][i] = 0.0;

  if (A.kind == K_FWD || A.kind == K_WHT) {
    for (int x = tid; x < N; x += SMALL_NT) sp[x] = load_val<T>(A.load_mode, in, x, nmask, l0cs, n);
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
    for (int x = tid; x < N; x += SMALL_NT) {
      store_val(A.store_mode, out, x, nmask, sp[x]);
      if (A.flags & F_ENERGY) red[tid][0] += (double)(sp[x] * sp[x] * table[x]);
    }
  } else if (A.kind == K_BWD) {
    const bool init = (A.flags & F_LAMBDA_INIT) != 0;
    for (int x = tid; x < N; x += SMALL_NT) {
      sp[x] = in[x];
      sl[x] = init ? table[x] * sp[x] : lin[x];
      if (A.flags & F_ENERGY) red[tid][SMALL_MAXN] += (double)(sp[x] * sl[x]);
    }
    __syncthreads();
    for (int b = 0; b < n; ++b) {
      if (!((gm >> b) & 1u)) continue;
      for (int pi = tid; pi < N / 2; pi += SMALL_NT) {
        const int x0 = ((pi >> b) << (b + 1)) | (pi & ((1 << b) - 1));
        const int x1 = x0 | (1 << b);
        red[tid][b] += (double)(sl[x1] * sp[x0] - sl[x0] * sp[x1]);
      }
    }
    __syncthreads();
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
    for (int x = tid; x < N; x += SMALL_NT) store_val(A.store_mode, out, x, nmask, sl[x]);
  } else if (A.kind == K_GRAD_L0) {
    const bool init = (A.flags & F_LAMBDA_INIT) != 0;
    for (int x = tid; x < N; x += SMALL_NT) {
      const T psi0 = product_state<T>(x, l0cs, n);
      const T lam = init ? table[x] * psi0 : lin[x];
      if (init) red[tid][SMALL_MAXN] += (double)(psi0 * lam);
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
      red[tid][SMALL_MAXN] += (double)(p * acc);
    }
  }
  __syncthreads();
  if (tid <= SMALL_MAXN) {
    double s = 0.0;
    for (int i = 0; i < SMALL_NT; ++i) s += red[i][tid];
    const int q = tid;
    if (q < SMALL_MAXN) {
      const bool want = (A.kind == K_BWD && ((gm >> q) & 1u)) || (A.kind == K_GRAD_L0 && q < n);
      if (want) part[(long long)q * A.tiles] = s;
    }
    if (A.kind == K_FWD && (A.flags & F_ENERGY) && q == 0) A.epart[job * A.part_stride] = s;
    if (q == SMALL_MAXN && (A.flags & F_ENERGY) && A.kind != K_FWD)
      A.epart[job * A.part_stride] = s;
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

// --------------------------------------------------------------- launchers --
int max_tile_bits(int prec) { return prec ? 13 : 14; }

size_t pass_smem_bytes(int prec, int kind, int tb) {
  const size_t es = prec ? 8 : 4;
  if (tb < 10) return 0;
  if (kind == K_BWD) return 2 * (es << tb);
  if (kind == K_FWD || kind == K_WHT) return es << tb;
  return 0;
}

template <typename T, int TB>
static cudaError_t launch_tb(const PassArgs &A, int jobs, int nterm, cudaStream_t s) {
  const dim3 grid((unsigned)A.tiles, (unsigned)jobs);
  const dim3 block(1 << (TB - 5));
  cudaError_t err = cudaSuccess;
  switch (A.kind) {
    case K_FWD:
    case K_WHT: {
      const size_t smem = sizeof(T) << TB;
      auto k = (A.kind == K_WHT) ? k_fwd<T, TB, true> : k_fwd<T, TB, false>;
      err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
      k<<<grid, block, smem, s>>>(A);
      break;
    }
    case K_BWD: {
      const size_t smem = 2 * (sizeof(T) << TB);
      err = cudaFuncSetAttribute(k_bwd<T, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
      k_bwd<T, TB><<<grid, block, smem, s>>>(A);
      break;
    }
    case K_GRAD_L0:
      k_grad_l0<T, TB><<<grid, block, 0, s>>>(A);
      break;
    case K_LAMBDA_XY: {
      const size_t smem = xy_layout(A.ngroups, nterm, (int)sizeof(T)).total;
      if (smem > 200 * 1024) return cudaErrorInvalidValue;
      err = cudaFuncSetAttribute(k_lambda_xy<T, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
      k_lambda_xy<T, TB><<<grid, block, smem, s>>>(A);
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

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
    case 13: return launch_tb<T, 13>(A, jobs, nterm, s);
    case 14:
      if constexpr (sizeof(T) == 4) return launch_tb<T, 14>(A, jobs, nterm, s);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pass(int prec, const PassArgs &A, int jobs, int nterm, cudaStream_t s) {
  if (jobs < 1 || A.tiles < 1) return cudaErrorInvalidValue;
  return prec ? launch_typed<double>(A, jobs, nterm, s) : launch_typed<float>(A, jobs, nterm, s);
}

size_t xy_smem_bytes(int prec, int ngroups, int nterm) {
  return xy_layout(ngroups, nterm, prec ? 8 : 4).total;
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
