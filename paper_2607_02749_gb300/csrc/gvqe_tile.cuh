// gvqe_tile.cuh -- the tile-pass kernels of the gvqe engine (templates).
//
// A CTA owns one tile of 2^TB real amplitudes; each of its 2^(TB-5) threads
// holds 32 amplitudes in registers at a time, and the tile moves through
// register "rounds".  In every round register bit 0 is tile bit 0, so a
// thread's elements 2m and 2m+1 are neighbours in shared and global memory and
// move as one 8-byte (FP32) or 16-byte (FP64) access:
//   round L: registers <-> tile bits 0, 6..9; lanes <-> bits 1..5; warps <->
//            bits 10..TB-1 (global loads/stores here are coalesced warp accesses)
//   round M: registers <-> tile bits 0..4 (16-byte vector shared-memory
//            accesses); lanes <-> bits 5..9
//   round H: registers <-> tile bits 0, 5, 10..TB-1 (and, for TB < 13, gate-free
//            group bits below 10); threads <-> bits 1..4, 6..9
// Rounds L and M of one warp cover the same 1024 tile amplitudes, so the L<->M
// transition only synchronises the warp; round H crosses warps.  RY gates on the
// bits held in registers are applied in registers (FP32: packed f32x2 FMAs on
// amplitude pairs, every gate but the one on tile bit 0); shared memory only
// transposes the tile between rounds.  The shared tile is swizzled (16-byte
// chunk index XOR the 128-byte row index) so all three access shapes are
// conflict-free.
//
// Global indices are 32-bit element offsets inside one state (n <= 30).
// Layout FULL: tile bits == global bits [0, TB) (the first pass of a layer,
// tile t covers elements [t 2^TB, (t+1) 2^TB)).  Layout STRIDED: tile bits
// [0, c) -> global [0, c), tile bits [c, TB) -> global [a, a + TB - c).
//
// Accumulation: energies and gradients sum one thread's products and one
// warp's lanes in the amplitude precision, then everything above a warp in
// FP64 in a fixed order (deterministic).
#pragma once
#include <cstdint>
#include <mutex>
#include <unordered_map>

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

// ------------------------------------------------------------- f32x2 ops --
__device__ __forceinline__ unsigned long long pk(float2 v) {
  return ((unsigned long long)__float_as_uint(v.y) << 32) | __float_as_uint(v.x);
}
__device__ __forceinline__ unsigned long long pk(float a, float b) {
  return ((unsigned long long)__float_as_uint(b) << 32) | __float_as_uint(a);
}
__device__ __forceinline__ float2 upk(unsigned long long r) {
  return make_float2(__uint_as_float((unsigned)r), __uint_as_float((unsigned)(r >> 32)));
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

// --------------------------------------------------------- register block --
// 32 amplitudes of one round; register bit j of the element index k is mapped
// to a tile bit by the round.
template <typename T>
struct Reg32;

// float: element k lives in v[k >> 1].x / .y, so register bits >= 1 pair whole
// float2 values and run as packed f32x2 arithmetic.
template <>
struct Reg32<float> {
  float2 v[16];
  __device__ __forceinline__ float get(int k) const { return (k & 1) ? v[k >> 1].y : v[k >> 1].x; }
  __device__ __forceinline__ float2 pair(int m) const { return v[m]; }
  __device__ __forceinline__ void set_pair(int m, float2 p) { v[m] = p; }
  __device__ __forceinline__ void set(int k, float x) {
    if (k & 1)
      v[k >> 1].y = x;
    else
      v[k >> 1].x = x;
  }
  // RY on register bit JB >= 1 with pre-packed coefficient pairs (c,c), (s,s), (-s,-s)
  template <int JB>
  __device__ __forceinline__ void rot_pk(unsigned long long c2, unsigned long long s2, unsigned long long ns2) {
    constexpr int B = 1 << (JB - 1);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      if (m & B) continue;
      const unsigned long long a = pk(v[m]), b = pk(v[m | B]);
      v[m] = upk(fma2(ns2, b, mul2(c2, a)));
      v[m | B] = upk(fma2(s2, a, mul2(c2, b)));
    }
  }
  // RY on register bit JB: (a, b) -> (c a - s b, s a + c b)
  template <int JB>
  __device__ __forceinline__ void rot(float c, float s) {
    if constexpr (JB == 0) {
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const float a = v[m].x, b = v[m].y;
        v[m].x = c * a - s * b;
        v[m].y = s * a + c * b;
      }
    } else {
      constexpr int B = 1 << (JB - 1);
      const unsigned long long c2 = pk(c, c), s2 = pk(s, s), ns2 = pk(-s, -s);
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        if (m & B) continue;
        const unsigned long long a = pk(v[m]), b = pk(v[m | B]);
        v[m] = upk(fma2(ns2, b, mul2(c2, a)));
        v[m | B] = upk(fma2(s2, a, mul2(c2, b)));
      }
    }
  }
  // unnormalised Walsh-Hadamard butterfly: (a, b) -> (a + b, a - b)
  template <int JB>
  __device__ __forceinline__ void wht() {
    if constexpr (JB == 0) {
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const float a = v[m].x, b = v[m].y;
        v[m].x = a + b;
        v[m].y = a - b;
      }
    } else {
      constexpr int B = 1 << (JB - 1);
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        if (m & B) continue;
        const unsigned long long a = pk(v[m]), b = pk(v[m | B]);
        v[m] = upk(add2(a, b));
        v[m | B] = upk(sub2(a, b));
      }
    }
  }
  // this = psi: sum over pairs (k0, k1 = k0 | bit) of lam[k1] psi[k0] - lam[k0] psi[k1]
  template <int JB>
  __device__ __forceinline__ float grad(const Reg32 &lam) const {
    if constexpr (JB == 0) {
      float acc = 0.f;
#pragma unroll
      for (int m = 0; m < 16; ++m) acc += lam.v[m].y * v[m].x - lam.v[m].x * v[m].y;
      return acc;
    } else {
      constexpr int B = 1 << (JB - 1);
      unsigned long long p[2] = {0, 0}, q[2] = {0, 0};
      int u = 0;
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        if (m & B) continue;
        p[u & 1] = fma2(pk(lam.v[m | B]), pk(v[m]), p[u & 1]);
        q[u & 1] = fma2(pk(lam.v[m]), pk(v[m | B]), q[u & 1]);
        ++u;
      }
      const float2 r = upk(sub2(add2(p[0], p[1]), add2(q[0], q[1])));
      return r.x + r.y;
    }
  }
};

template <>
struct Reg32<double> {
  double v[32];
  __device__ __forceinline__ double get(int k) const { return v[k]; }
  __device__ __forceinline__ void set(int k, double x) { v[k] = x; }
  __device__ __forceinline__ double2 pair(int m) const { return make_double2(v[2 * m], v[2 * m + 1]); }
  __device__ __forceinline__ void set_pair(int m, double2 p) {
    v[2 * m] = p.x;
    v[2 * m + 1] = p.y;
  }
  template <int JB>
  __device__ __forceinline__ void rot(double c, double s) {
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      if (k & (1 << JB)) continue;
      const double a = v[k], b = v[k | (1 << JB)];
      v[k] = c * a - s * b;
      v[k | (1 << JB)] = s * a + c * b;
    }
  }
  template <int JB>
  __device__ __forceinline__ void wht() {
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      if (k & (1 << JB)) continue;
      const double a = v[k], b = v[k | (1 << JB)];
      v[k] = a + b;
      v[k | (1 << JB)] = a - b;
    }
  }
  template <int JB>
  __device__ __forceinline__ double grad(const Reg32 &lam) const {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      if (k & (1 << JB)) continue;
      acc += lam.v[k | (1 << JB)] * v[k] - lam.v[k] * v[k | (1 << JB)];
    }
    return acc;
  }
};

// ----------------------------------------------------------------- helpers --
template <typename T>
__device__ __forceinline__ int swz(int i) {
  constexpr int CH = 16 / (int)sizeof(T);  // amplitudes per 16-byte chunk
  return i ^ (((i >> 5) & 7) * CH);
}

// Launch order of tiles: block bx runs tile t; with pair_mask != 0 the tiles t and
// t ^ pair_mask (whose gathers read the two halves of the same sectors) run next
// to each other: block 2u + b runs tile u' ^ (b ? pair_mask : 0), u' = u with a 0
// inserted at the highest bit of pair_mask.
__device__ __forceinline__ uint32_t tile_of_block(uint32_t bx, uint32_t tiles, uint32_t pair_mask) {
  if (pair_mask == 0 || tiles < 2) return bx;
  const int hb = 31 - __clz(pair_mask);
  const uint32_t v = bx >> 1;
  const uint32_t u = ((v >> hb) << (hb + 1)) | (v & ((1u << hb) - 1u));
  return (bx & 1) ? (u ^ pair_mask) : u;
}

// Global offset of tile t: its index bits fill the global bits outside the
// tile in increasing order, [c, a), then [a + k1, a + k1 + gap) (split layout),
// then [a + gap + tb - c, n).
__device__ __forceinline__ uint32_t tile_base(uint32_t t, const PassArgs &A, int tb) {
  const int lo = A.a - A.c;
  const uint32_t t0 = t & ((1u << lo) - 1);
  const uint32_t tm = (t >> lo) & ((1u << A.gap) - 1);
  const uint32_t th = t >> (lo + A.gap);
  return (t0 << A.c) | (tm << (A.a + A.k1)) | (th << (A.a + A.gap + tb - A.c));
}


template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// c, negated when bit is 1 (a sign-bit flip, no branch).
__device__ __forceinline__ float flip_sign(float c, uint32_t bit) {
  return __int_as_float(__float_as_int(c) ^ (int)(bit << 31));
}
__device__ __forceinline__ double flip_sign(double c, uint32_t bit) {
  return __longlong_as_double(__double_as_longlong(c) ^ ((long long)bit << 63));
}

// Global offset of a tile bit under the STRIDED layout.
__device__ __forceinline__ uint32_t gbit(int t, const PassArgs &A) { return 1u << tile_gbit(t, A.c, A.a, A.k1, A.gap); }
// Global offset (within its tile) of tile index i under the STRIDED layout.
__device__ __forceinline__ uint32_t tile_goff(uint32_t i, const PassArgs &A) {
  const uint32_t hi = i >> A.c;
  return (i & ((1u << A.c) - 1)) + ((hi & ((1u << A.k1) - 1)) << A.a) + ((hi >> A.k1) << (A.a + A.k1 + A.gap));
}

// Gate coefficients of one pass, per tile bit: (cos, sin) and, for FP32, the
// packed pairs (c,c), (s,s), (-s,-s) the f32x2 rotations take, built once per CTA.
template <typename T2>
struct GateTab {
  T2 cs[16];
  unsigned long long c2[16], s2[16], ns2[16];
  __device__ __forceinline__ void pack(int tid) {
    if (tid < 16) {
      const float c = (float)cs[tid].x, s = (float)cs[tid].y;
      c2[tid] = pk(c, c);
      s2[tid] = pk(s, s);
      ns2[tid] = pk(-s, -s);
    }
  }
};

// PACKED: FP32 rotations take the pre-packed pairs of the table (fewer registers
// live when false: the pairs are packed at the call).
template <int NB, bool WHT, bool PACKED = true, int RO = 0, typename T, typename T2>
__device__ __forceinline__ void round_gates(Reg32<T> &r, const GateTab<T2> &gt, uint32_t gmask, int tbit0,
                                            bool inverse) {
  // register bit RO + j holds tile bit tbit0 + j; RY(theta), or RY(-theta) when inverse
#define GVQE_GATE(J)                                                                       \
  if (NB > J && ((gmask >> (tbit0 + J)) & 1u)) {                                           \
    if (WHT) {                                                                             \
      r.template wht<J + RO>();                                                            \
    } else if constexpr (PACKED && sizeof(T) == 4 && J + RO > 0) {                         \
      const int tb_ = tbit0 + J;                                                           \
      r.template rot_pk<(J + RO > 0 ? J + RO : 1)>(gt.c2[tb_], inverse ? gt.ns2[tb_] : gt.s2[tb_], \
                                                   inverse ? gt.s2[tb_] : gt.ns2[tb_]);   \
    } else {                                                                               \
      const T2 cs = gt.cs[tbit0 + J];                                                      \
      r.template rot<J + RO>(cs.x, inverse ? -cs.y : cs.y);                                \
    }                                                                                      \
  }
  GVQE_GATE(0)
  GVQE_GATE(1)
  GVQE_GATE(2)
  GVQE_GATE(3)
  GVQE_GATE(4)
#undef GVQE_GATE
}

// Gradient partials of one round: the (up to 5, padded to 8) per-thread sums are
// reduced over the warp with a transposed butterfly (each exchange halves the
// values a lane carries), then lane (j << 2) holds value j and stores it.
// X5: also the gate of tile bit 5 on register bit 1 (round H), in slot 5.
// The warp partial is stored in the working precision T; the tile epilogue
// converts it to FP64 (exactly) and sums the warps in FP64, so the narrow FP64
// pipe sees one warp's adds per tile instead of a conversion in every warp
// after every round.
template <int NB, int RO = 0, bool X5 = false, typename T>
__device__ __forceinline__ void round_grads(const Reg32<T> &psi, const Reg32<T> &lam, uint32_t gmask, int tbit0,
                                            T *wred, int lane) {
  T v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = T(0);
  if (X5 && ((gmask >> 5) & 1u)) v[5] = psi.template grad<1>(lam);
#define GVQE_GV(J)                                          \
  if (NB > J && ((gmask >> (tbit0 + J)) & 1u)) {            \
    constexpr int JB_ = (J + RO < 5 ? J + RO : 4);          \
    v[J] = psi.template grad<JB_>(lam);                     \
  }
  GVQE_GV(0)
  GVQE_GV(1)
  GVQE_GV(2)
  GVQE_GV(3)
  GVQE_GV(4)
#undef GVQE_GV
  // stage 1: lanes with bit 4 set keep values 4..7, the others 0..3
  const bool b4 = (lane >> 4) & 1;
  T u[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const T mine = b4 ? v[4 + j] : v[j];
    const T other = b4 ? v[j] : v[4 + j];
    u[j] = mine + __shfl_xor_sync(0xffffffffu, other, 16);
  }
  const bool b3 = (lane >> 3) & 1;
  T t2[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const T mine = b3 ? u[2 + j] : u[j];
    const T other = b3 ? u[j] : u[2 + j];
    t2[j] = mine + __shfl_xor_sync(0xffffffffu, other, 8);
  }
  const bool b2 = (lane >> 2) & 1;
  T r = (b2 ? t2[1] : t2[0]) + __shfl_xor_sync(0xffffffffu, b2 ? t2[0] : t2[1], 4);
  r += __shfl_xor_sync(0xffffffffu, r, 2);
  r += __shfl_xor_sync(0xffffffffu, r, 1);
  // lane holds value index (b4 << 2) | (b3 << 1) | b2
  if ((lane & 3) == 0) {
    const int j = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    if (j < NB && ((gmask >> (tbit0 + j)) & 1u))
      wred[tbit0 + j] = r;
    else if (X5 && j == 5 && ((gmask >> 5) & 1u))
      wred[5] = r;
  }
}

// Complex path, round L: RZ gradients Im<lam|Z_q|psi> = sum_x s_q(x) w(x) with
// w = Im(conj(lam) psi) and s_q = +1 (x_q = 0) or -1, for every gate bit of the
// tile: register bits (tile bits 6..9) give signed sums over the thread's
// pairs, lane bits (1..5) sign the thread total, warp bits (10..) sign the warp
// total.  The 16 per-tile-bit values go through one transposed warp butterfly;
// wredz[tile bit] receives the warp's partial.
template <typename T>
__device__ __forceinline__ void rz_grads_L(const Reg32<T> &psi, const Reg32<T> &lam, uint32_t gmask, T *wredz,
                                           int lane, int w) {
  T tot = T(0), d[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const auto l = lam.pair(m), p = psi.pair(m);
    const T x = l.x * p.y - l.y * p.x;
    tot += x;
#pragma unroll
    for (int j = 0; j < 4; ++j) d[j] += ((m >> j) & 1) ? -x : x;
  }
  T v[16];
#pragma unroll
  for (int b = 0; b < 16; ++b) {
    if (b >= 1 && b <= 5)
      v[b] = ((lane >> (b - 1)) & 1) ? -tot : tot;
    else if (b >= 6 && b <= 9)
      v[b] = d[b - 6];
    else if (b >= 10)
      v[b] = tot;
    else
      v[b] = T(0);
  }
  // transposed butterfly: each exchange halves the values a lane carries
  T u8[8], u4[4], u2[2];
  const bool b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1, b1 = (lane >> 1) & 1;
#pragma unroll
  for (int j = 0; j < 8; ++j)
    u8[j] = (b4 ? v[8 + j] : v[j]) + __shfl_xor_sync(0xffffffffu, b4 ? v[j] : v[8 + j], 16);
#pragma unroll
  for (int j = 0; j < 4; ++j)
    u4[j] = (b3 ? u8[4 + j] : u8[j]) + __shfl_xor_sync(0xffffffffu, b3 ? u8[j] : u8[4 + j], 8);
#pragma unroll
  for (int j = 0; j < 2; ++j)
    u2[j] = (b2 ? u4[2 + j] : u4[j]) + __shfl_xor_sync(0xffffffffu, b2 ? u4[j] : u4[2 + j], 4);
  T r = (b1 ? u2[1] : u2[0]) + __shfl_xor_sync(0xffffffffu, b1 ? u2[0] : u2[1], 2);
  r += __shfl_xor_sync(0xffffffffu, r, 1);
  if ((lane & 1) == 0) {
    const int b = (b4 ? 8 : 0) + (b3 ? 4 : 0) + (b2 ? 2 : 0) + (b1 ? 1 : 0);
    if ((gmask >> b) & 1u) {
      wredz[b] = (b >= 10 && ((w >> (b - 10)) & 1)) ? -r : r;
    }
  }
}

// --------------------------------------------------- shared-memory rounds --
// In every round register bit 0 holds tile bit 0, so a thread's elements
// 2m and 2m+1 are neighbours in the tile and in global memory: rounds L and H
// move them as one 8-byte (FP32) or 16-byte (FP64) access.
//
// Round L: element k = 2m + e of thread (lane, warp w) is tile index
// e + 2 lane + 64 m + 1024 w: register bits 1..4 hold tile bits 6..9, the lane
// tile bits 1..5, the warp tile bits 10...
__device__ __forceinline__ int idx_L(int lane, int w, int m) { return (lane << 1) + (m << 6) + (w << 10); }

// Per-thread parts of the swizzled round-L and round-H offsets.  The swizzle
// XORs tile bits 2..4 (FP32; 1..3 for FP64) with tile bits 5..7, and in both
// layouts the XORed bits come from the thread index alone while bits 5..7 come
// from the thread index and at most two pair-index bits.  So pair m of round L
// sits at L[m & 3] + 64 m and pair m of round H at H[m & 3] + idx_H_pair(m):
// a few per-thread bases plus compile-time offsets.
struct SBase {
  int L[4];
  int H[4];
};
template <int TB>
__device__ __forceinline__ int idx_H_thread(int tid);
template <int TB, typename T>
__device__ __forceinline__ SBase sbase(int tid) {
  constexpr int CH = 16 / (int)sizeof(T);
  const int lane = tid & 31, w = tid >> 5;
  SBase b;
#pragma unroll
  for (int j = 0; j < 4; ++j) b.L[j] = ((lane << 1) ^ ((((lane >> 4) & 1) | (j << 1)) * CH)) + (w << 10);
  const int thr = idx_H_thread<TB>(tid);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int b7 = TB >= 11 ? ((tid >> 5) & 1) : ((j >> 1) & 1);  // tile bit 7: thread bit 5 or pair bit 1
    b.H[j] = thr ^ (((j & 1) | (((tid >> 4) & 1) << 1) | (b7 << 2)) * CH);
  }
  return b;
}
template <typename T>
__device__ __forceinline__ void sts_L(T *s, const SBase &sb, const Reg32<T> &r) {
  using T2 = typename V2<T>::type;
#pragma unroll
  for (int m = 0; m < ROUND / 2; ++m) *reinterpret_cast<T2 *>(s + sb.L[m & 3] + (m << 6)) = r.pair(m);
}
template <typename T>
__device__ __forceinline__ void lds_L(const T *s, const SBase &sb, Reg32<T> &r) {
  using T2 = typename V2<T>::type;
#pragma unroll
  for (int m = 0; m < ROUND / 2; ++m) r.set_pair(m, *reinterpret_cast<const T2 *>(s + sb.L[m & 3] + (m << 6)));
}
// Round M: group G's 32 consecutive amplitudes (register bits 0..4 = tile
// bits 0..4) as 16-byte chunks in swizzled order.
__device__ __forceinline__ void lds_M(const float *s, int G, Reg32<float> &r) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float4 q = *reinterpret_cast<const float4 *>(s + (G << 5) + ((c ^ (G & 7)) << 2));
    r.v[2 * c] = make_float2(q.x, q.y);
    r.v[2 * c + 1] = make_float2(q.z, q.w);
  }
}
__device__ __forceinline__ void sts_M(float *s, int G, const Reg32<float> &r) {
#pragma unroll
  for (int c = 0; c < 8; ++c)
    *reinterpret_cast<float4 *>(s + (G << 5) + ((c ^ (G & 7)) << 2)) =
        make_float4(r.v[2 * c].x, r.v[2 * c].y, r.v[2 * c + 1].x, r.v[2 * c + 1].y);
}
__device__ __forceinline__ void lds_M(const double *s, int G, Reg32<double> &r) {
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const double2 q = *reinterpret_cast<const double2 *>(s + (G << 5) + ((c ^ (G & 7)) << 1));
    r.v[2 * c] = q.x;
    r.v[2 * c + 1] = q.y;
  }
}
__device__ __forceinline__ void sts_M(double *s, int G, const Reg32<double> &r) {
#pragma unroll
  for (int c = 0; c < 16; ++c)
    *reinterpret_cast<double2 *>(s + (G << 5) + ((c ^ (G & 7)) << 1)) = make_double2(r.v[2 * c], r.v[2 * c + 1]);
}
// Round H: element k = 2m + e of thread tid is tile index e + idx_H(tid, m).
// Register bit 1 holds tile bit 5, register bits 2..1+H tile bits 10..TB-1
// (H = TB - 10) and the remaining register bits tile bits TB-3..9; the thread
// index covers tile bits 1..4 (its low four bits) and 6.. (the rest).  Only
// register bits 1..1+H carry gates here: tile bit 5 and the high tile bits.
template <int TB>
__device__ __forceinline__ int idx_H_thread(int tid) { return ((tid & 15) << 1) | ((tid >> 4) << 6); }
template <int TB>
__host__ __device__ constexpr int tbit_H(int j) {  // tile bit of pair-index bit j (register bit j + 1)
  return j == 0 ? 5 : (j <= TB - 10 ? 9 + j : TB - 3 + (j - 1 - (TB - 10)));
}
template <int TB>
__device__ __forceinline__ int idx_H_pair(int m) {
  int o = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) o |= ((m >> j) & 1) << tbit_H<TB>(j);
  return o;
}
template <int TB, typename T>
__device__ __forceinline__ void lds_H(const T *s, const SBase &sb, Reg32<T> &r) {
  using T2 = typename V2<T>::type;
#pragma unroll
  for (int m = 0; m < ROUND / 2; ++m)
    r.set_pair(m, *reinterpret_cast<const T2 *>(s + sb.H[m & 3] + idx_H_pair<TB>(m)));
}
template <int TB, typename T>
__device__ __forceinline__ void sts_H(T *s, const SBase &sb, const Reg32<T> &r) {
  using T2 = typename V2<T>::type;
#pragma unroll
  for (int m = 0; m < ROUND / 2; ++m) *reinterpret_cast<T2 *>(s + sb.H[m & 3] + idx_H_pair<TB>(m)) = r.pair(m);
}

// Gray-code order of the 16 element pairs: consecutive pairs differ in one
// pair-index bit, so a strided global offset advances by one add.
__host__ __device__ constexpr int gray(int k) { return k ^ (k >> 1); }
__host__ __device__ constexpr int gray_bit(int k) {  // bit flipped between gray(k-1) and gray(k)
  return (k & 1) ? 0 : (k & 2) ? 1 : (k & 4) ? 2 : 3;
}

// Global element offsets of a thread's round-L and round-H pairs.  Tile bit
// 0 is global bit 0 in both layouts (the STRIDED carry is at least 3), so
// element 2m + 1 sits right after element 2m.
template <int TB, bool FULL>
struct GIdx {
  uint32_t baseL;  // offset of pair 0 in round L
  uint32_t SL[4];  // offset of pair-index bit j in round L (tile bit 6 + j)
  uint32_t baseH;  // offset of pair 0 in round H
  uint32_t SH[4];  // offset of pair-index bit j in round H (tile bit tbit_H(j))
  __device__ __forceinline__ void init(uint32_t tbase, const PassArgs &A, int lane, int w, int tid) {
    const uint32_t iL = (uint32_t)idx_L(lane, w, 0), iH = (uint32_t)idx_H_thread<TB>(tid);
    baseL = tbase + (FULL ? iL : tile_goff(iL, A));
    baseH = tbase + (FULL ? iH : tile_goff(iH, A));
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      SL[j] = FULL ? (1u << (6 + j)) : gbit(6 + j, A);
      SH[j] = FULL ? (1u << tbit_H<TB>(j)) : gbit(tbit_H<TB>(j), A);
    }
  }
};

// Visit a thread's 16 element pairs of round L (or H): f(m, global offset of element 2m).
template <typename F>
__device__ __forceinline__ void for_pairs(uint32_t base, const uint32_t (&S)[4], F &&f) {
  uint32_t o = base;
#pragma unroll
  for (int k = 0; k < ROUND / 2; ++k) {
    const int m = gray(k);
    if (k > 0) {
      const int j = gray_bit(k);
      o = ((m >> j) & 1) ? o + S[j] : o - S[j];
    }
    f(m, o);
  }
}
template <int TB, bool FULL, typename F>
__device__ __forceinline__ void for_L(const GIdx<TB, FULL> &gi, F &&f) {
  for_pairs(gi.baseL, gi.SL, f);
}
// Round-L pairs of a FULL-layout pass through the entangler map: f(m, x) with
// x = A^-1 y of element 2m.  A^-1 is GF(2)-linear and the Gray-code walk flips
// one bit of y per step, so x advances by one XOR with that bit's image.
template <int TB, typename F>
__device__ __forceinline__ void for_L_ent(const GIdx<TB, true> &gi, uint32_t nmask, const EntMap &em, int n, F &&f) {
  uint32_t d[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) d[j] = ent_inv(gi.SL[j], nmask, em, n);
  uint32_t x = ent_inv(gi.baseL, nmask, em, n);
#pragma unroll
  for (int k = 0; k < ROUND / 2; ++k) {
    const int m = gray(k);
    if (k > 0) x ^= d[gray_bit(k)];
    f(m, x);
  }
}
template <int TB, bool FULL, typename F>
__device__ __forceinline__ void for_H(const GIdx<TB, FULL> &gi, F &&f) {
  for_pairs(gi.baseH, gi.SH, f);
}

template <typename T2>
__device__ __forceinline__ void load_gate_coeffs(const PassArgs &A, const T2 *cs, T2 *gcs, int tid) {
  if (tid < 16) {
    T2 v;
    v.x = 1;
    v.y = 0;
    if (tid < A.tb && ((A.gate_mask >> tid) & 1u)) {
      const int q = tile_gbit(tid, A.c, A.a, A.k1, A.gap);
      v = cs[A.layer * A.pstride + q - A.qoff];
    }
    gcs[tid] = v;
  }
}

// ------------------------------------------------ EfficientSU2 (complex) --
// With the full EfficientSU2 rotation layer (RY, then RZ on every qubit) the
// state is complex.  It is stored as 2^(n+1) reals, u[2x] = Re psi(x) and
// u[2x + 1] = Im psi(x): index bit 0 is the real/imaginary channel and index
// bit q + 1 is qubit q, so a register pair (tile bit 0) is one amplitude.  RY
// and the CX permutations act alike on both channels; RZ(theta) on qubit q
// multiplies psi(x) by exp(-i theta/2) when x_q = 0 and exp(+i theta/2) when
// x_q = 1.  A pass applies its qubits' RZ after their RY (they commute with the
// other qubits' gates) as one phase per amplitude: the product of the thread's
// tile bits' factors and of the register bits' factors.  The forward pass applies
// it in round H (preg), the backward pass takes it off psi and lambda in round L
// (pregL), before the RY gradients and RY(-theta).

template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b) {
  T2 r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename T2>
__device__ __forceinline__ T2 cconj(T2 a) {
  a.y = -a.y;
  return a;
}

template <typename T2, int TB>
struct SU2Tab {
  T2 zh[16];    // per tile bit: (cos, sin) of theta_z / 2, (1, 0) without an RZ
  T2 preg[16];  // round H: the phase of register pattern m
  T2 pregL[16]; // round L: the phase of register pattern m (tile bits 6..9)
  // threads 0..15; the caller synchronises before use
  __device__ __forceinline__ void build(const PassArgs &A, const T2 *cs, int tid) {
    if (tid >= 16) return;
    auto half = [&](int tb) {
      T2 v;
      v.x = 1;
      v.y = 0;
      if (tb < A.tb && ((A.gate_mask >> tb) & 1u)) {
        const int g = tile_gbit(tb, A.c, A.a, A.k1, A.gap);
        v = cs[A.layer * A.pstride + A.zoff + g - A.qoff];
      }
      return v;
    };
    const T2 h = half(tid);
    zh[tid] = h;
    T2 p;
    p.x = 1;
    p.y = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {  // pair-index bit j holds tile bit tbit_H(j)
      T2 e = half(tbit_H<TB>(j));
      if (!((tid >> j) & 1)) e.y = -e.y;  // x_q = 0: exp(-i theta/2)
      p = cmul(p, e);
    }
    preg[tid] = p;
    T2 q;
    q.x = 1;
    q.y = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {  // round L: pair-index bit j holds tile bit 6 + j
      T2 e = half(6 + j);
      if (!((tid >> j) & 1)) e.y = -e.y;
      q = cmul(q, e);
    }
    pregL[tid] = q;
  }
  // phase of this thread's round-L tile bits (lanes: 1..5, warps: 10..)
  __device__ __forceinline__ T2 thread_phase_L(int lane, int w) const {
    T2 p;
    p.x = 1;
    p.y = 0;
#pragma unroll
    for (int b = 1; b < TB; ++b) {
      if (b >= 6 && b <= 9) continue;
      const int bit = b <= 5 ? ((lane >> (b - 1)) & 1) : ((w >> (b - 10)) & 1);
      T2 e = zh[b];
      if (!bit) e.y = -e.y;
      p = cmul(p, e);
    }
    return p;
  }
  // phase of this thread's round-H tile bits (those not in its registers)
  __device__ __forceinline__ T2 thread_phase(int tid) const {
    const int base = idx_H_thread<TB>(tid);
    T2 p;
    p.x = 1;
    p.y = 0;
#pragma unroll
    for (int b = 1; b < TB; ++b) {
      if (b == tbit_H<TB>(0) || b == tbit_H<TB>(1) || b == tbit_H<TB>(2) || b == tbit_H<TB>(3)) continue;
      T2 e = zh[b];
      if (!((base >> b) & 1)) e.y = -e.y;
      p = cmul(p, e);
    }
    return p;
  }
};

// psi -> psi * phase (forward) or lambda -> lambda * conj(phase) (backward), round H
template <bool CONJ, typename T, typename T2, int TB>
__device__ __forceinline__ void apply_su2_phase(Reg32<T> &r, const SU2Tab<T2, TB> &zt, T2 pthr) {
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    T2 ph = cmul(pthr, zt.preg[m]);
    if (CONJ) ph = cconj(ph);
    r.set_pair(m, cmul(r.pair(m), ph));
  }
}

// Layer-0 product state psi_0(x) = prod_q f_q(x_q), f(0) = cos(t/2), f(1) = sin(t/2), tabulated
// per tile: bits 0..6 (lo), bits 7..TB (mid), the tile's bits above TB (hi, two values).
template <typename T, typename T2, int TB>
struct L0Tables {
  T lo[128];   // x bits 0..6
  T mid[128];  // x bits 7..TB
  T hi[2];     // x bits above TB
  // Across one tile x = xbase ^ (a linear image of the tile's y bits): the bits
  // above TB take two values, told apart by x bit kbit, and differ in hflip.
  __device__ __forceinline__ void build(const T2 *l0, int n, uint32_t xbase, int kbit, uint32_t hflip, int tid,
                                        int nthreads) {
    for (int m = tid; m < 256; m += nthreads) {
      const int hi7 = m >> 7, mm = m & 127;
      T p = T(1);
      const int q0 = hi7 ? 7 : 0;
      const int q1 = hi7 ? TB + 1 : 7;
      for (int q = q0; q < q1 && q < n; ++q) p *= ((mm >> (q - q0)) & 1) ? l0[q].y : l0[q].x;
      if (hi7)
        mid[mm] = p;
      else
        lo[mm] = p;
    }
    if (tid < 2) {
      T p = T(1);
      const uint32_t xh = xbase ^ ((((uint32_t)tid ^ (xbase >> kbit)) & 1u) ? hflip : 0u);
      for (int q = TB + 1; q < n; ++q) p *= ((xh >> q) & 1) ? l0[q].y : l0[q].x;
      hi[tid] = p;
    }
  }
  __device__ __forceinline__ T operator()(uint32_t x, int kbit) const {
    return lo[x & 127] * mid[(x >> 7) & ((1u << (TB - 6)) - 1)] * hi[(x >> kbit) & 1];
  }
};

// ------------------------------------------------------ forward tile pass --
// One tile of a forward pass: tile block index tb_idx of job `job` (the pairing
// of tiles H and ~H for gathering passes is applied here).  State loads go
// through L2 (ld.global.cg), so data written by other SMs is never read stale.
template <typename T, int TB, bool FULL, int LOAD, bool WHT, bool REUSE = true, bool CPLX = false>
__device__ __forceinline__ void fwd_tile(const PassArgs &A, int job, uint32_t tb_idx) {
  using T2 = typename V2<T>::type;
  constexpr int NT = 1 << (TB - 5);
  constexpr int NW = NT / 32;
  constexpr int H = TB - 10;
  constexpr bool L0 = (LOAD == LD_L0 || LOAD == LD_L0_GATHER);
  static_assert(!CPLX || (!L0 && !WHT), "the complex path starts from |0> and has no table build");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *s = reinterpret_cast<T *>(smem_raw);
  __shared__ GateTab<T2> gt;
  __shared__ double ered[NW];
  __shared__ L0Tables<T, T2, TB> tab;
  __shared__ SU2Tab<T2, TB> zt;

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const SBase sb = sbase<TB, T>(tid);
  const uint32_t t = tile_of_block(tb_idx, (uint32_t)A.tiles, A.pair_mask);
  const uint32_t tbase = tile_base(t, A, TB);
  const uint32_t nmask = (A.n >= 32) ? 0xffffffffu : ((1u << A.n) - 1);
  const uint32_t d1 = ent_inv(1u, nmask, A.em, A.n);  // the pair (y, y + 1) maps to (x, x ^ d1)
  const T2 *cs = reinterpret_cast<const T2 *>(A.cs) + (size_t)(A.job0 + job) * A.P;
  if (!WHT) {
    load_gate_coeffs(A, cs, gt.cs, tid);
  }
  if constexpr (CPLX) zt.build(A, cs, tid);
  if constexpr (L0) {
    const uint32_t xbase = (LOAD == LD_L0_GATHER) ? ent_inv(tbase, nmask, A.em, A.n) : tbase;
    const uint32_t hflip = (LOAD == LD_L0_GATHER) ? A.l0_hflip : 0u;
    tab.build(cs, A.n, xbase, A.l0_kbit, hflip, tid, NT);
  }
  const T *in = reinterpret_cast<const T *>(A.in) + (size_t)job * A.in_stride;
  T *out = reinterpret_cast<T *>(A.out) + (size_t)job * A.out_stride;
  const uint32_t gm = A.gate_mask;
  GIdx<TB, FULL> gi;
  gi.init(tbase, A, lane, w, tid);

  Reg32<T> r;
  // round L: global -> registers (tile bits 6..9) -> gates -> shared.  The
  // inverse CX chain maps the pair (y, y + 1) to (x, x ^ 3), x = A^-1 y.
  // State loads do not depend on the gate coefficients, so they are issued
  // before the barrier that publishes them and are in flight while the
  // coefficient loads complete; the layer-0 forms read the tables built above
  // and come after it.
  auto load_L = [&]() {
    if constexpr (FULL && (LOAD == LD_GATHER || LOAD == LD_L0_GATHER)) {
      const int kbit = A.l0_kbit;
      for_L_ent(gi, nmask, A.em, A.n, [&](int m, uint32_t x) {
        T2 v;
        if constexpr (LOAD == LD_GATHER && CPLX) {
          // the map keeps the channel bit: (re, im) of x stay neighbours
          v = __ldcg(reinterpret_cast<const T2 *>(in + x));
        } else if constexpr (LOAD == LD_GATHER) {
          v.x = __ldcg(in + x);
          v.y = __ldcg(in + (x ^ d1));
        } else {
          v.x = tab(x, kbit);
          v.y = tab(x ^ d1, kbit);
        }
        r.set_pair(m, v);
      });
    } else {
      for_L(gi, [&](int m, uint32_t y) {
        T2 v;
        if constexpr (LOAD == LD_PLAIN) {
          v = __ldcg(reinterpret_cast<const T2 *>(in + y));
        } else if constexpr (LOAD == LD_ZERO) {
          v.x = (y == 0) ? T(1) : T(0);
          v.y = T(0);
        } else {
          v.x = tab(y, TB);
          v.y = tab(y + 1, TB);
        }
        r.set_pair(m, v);
      });
    }
  };
  if constexpr (!L0) load_L();
  __syncthreads();
  if constexpr (L0) load_L();
  round_gates<4, WHT, false, 1>(r, gt, gm, 6, false);
  sts_L(s, sb, r);
  // round M: tile bits 0..4.  Layouts L and M of warp w both cover tile
  // amplitudes [1024 w, 1024 w + 1024), so the warp only syncs with itself.
  if (gm & 0x1Fu) {
    __syncwarp();
    lds_M(s, tid, r);
    round_gates<5, WHT, false>(r, gt, gm, 0, false);
    sts_M(s, tid, r);
  }
  __syncthreads();
  // round H: tile bits 5 and 10..TB-1, then the store and the energy epilogue
  lds_H<TB>(s, sb, r);
  round_gates<1, WHT, false, 1>(r, gt, gm, 5, false);
  round_gates<H, WHT, false, 2>(r, gt, gm, 10, false);
  if constexpr (CPLX) apply_su2_phase<false>(r, zt, zt.thread_phase(tid));
  const T *table = reinterpret_cast<const T *>(A.table) + (size_t)job * A.table_stride;
  const bool store = A.store_mode != ST_NONE;
  const bool energy = (A.flags & F_ENERGY) != 0;
  T eacc = T(0);
  if (!energy) {
    for_H(gi, [&](int m, uint32_t y) { *reinterpret_cast<T2 *>(out + y) = r.pair(m); });
  } else {
    for_H(gi, [&](int m, uint32_t y) {
      const T2 v = r.pair(m);
      if (store) *reinterpret_cast<T2 *>(out + y) = v;
      eacc += v.x * v.x * table[y] + v.y * v.y * table[y + 1];
    });
  }
  if (energy) {
    eacc = warp_sum(eacc);
    if (lane == 0) ered[w] = (double)eacc;
    __syncthreads();
    if (tid == 0) {
      double e = 0.0;
#pragma unroll
      for (int ww = 0; ww < NW; ++ww) e += ered[ww];
      A.epart[(size_t)job * A.part_stride + t] = e;
    }
  }
  if (REUSE) __syncthreads();  // shared tile and coefficients free for the caller's next tile
}

template <typename T, int TB, bool FULL, int LOAD, bool WHT, bool CPLX = false>
__global__ void __launch_bounds__(1 << (TB - 5), (TB <= 12 ? 8 : 4) / (sizeof(T) == 8 ? 2 : 1))
k_fwd(const PassArgs A) {
  fwd_tile<T, TB, FULL, LOAD, WHT, false, CPLX>(A, blockIdx.y, blockIdx.x);
}

// ------------------------------------------------------ backward tile pass --
// Asynchronous 16-byte global -> shared copies (L1 bypassed).
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Persistent CTAs walk the tiles blockIdx.x, +gridDim.x, ...  Each CTA owns
// two tile-sized shared buffers, one for psi and one for lambda.  The next
// tile's psi streams into the psi buffer once round H has read this tile's psi
// (it overlaps the rest of the lambda rounds and the store), and each warp
// refills its own part of the lambda buffer once its final round L has read it.
// Three CTAs share an SM: against three buffers at two CTAs per SM the extra
// warps hide more of the shared-memory round latency than the shorter lambda
// prefetch exposes.
//
// lambda and psi are both at the point right after this pass's gates.  Rounds
// L, M, H read both and form the gradients (all at that same point); round H
// then applies RY(-theta) to lambda on its bits, rounds M and L follow on
// theirs, and round L writes lambda (through the inverse CX chain for the
// first pass of a layer, layout FULL).  Gradient and energy partials are
// written per tile.
template <typename T, int TB, bool FULL, bool CPLX = false>
__global__ void __launch_bounds__(1 << (TB - 5), 3)
k_bwd(const PassArgs A) {
  using T2 = typename V2<T>::type;
  constexpr int NT = 1 << (TB - 5);
  constexpr int NW = NT / 32;
  constexpr int H = TB - 10;
  constexpr int TILE = 1 << TB;
  constexpr int CH = 16 / (int)sizeof(T);  // amplitudes per 16-byte chunk
  constexpr int CPT = TILE / CH / NT;      // chunks per thread per array
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *buf = reinterpret_cast<T *>(smem_raw);  // psi tile, lambda tile
  __shared__ GateTab<T2> gt;
  __shared__ T gred[2][NW][16];   // by tile parity: a warp may start the next
  __shared__ double ered[2][NW];  // tile while warp 0 still sums this one
  __shared__ T gredz[CPLX ? 2 : 1][CPLX ? NW : 1][16];  // complex path: RZ partials
  __shared__ SU2Tab<T2, TB> zt;

  const int job = blockIdx.y;
  if (A.minlayer != nullptr && !(A.flags & F_ENERGY) && A.layer < A.minlayer[A.job0 + job]) return;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const SBase sb = sbase<TB, T>(tid);
  const uint32_t tiles = (uint32_t)A.tiles;
  const uint32_t pair = A.pair_mask;
  const uint32_t nmask = (1u << A.n) - 1;
  const uint32_t d1 = ent_inv(1u, nmask, A.em, A.n);  // the pair (y, y + 1) maps to (x, x ^ d1)
  const T2 *cs = reinterpret_cast<const T2 *>(A.cs) + (size_t)(A.job0 + job) * A.P;
  load_gate_coeffs(A, cs, gt.cs, tid);
  if (sizeof(T) == 4) gt.pack(tid);
  if constexpr (CPLX) zt.build(A, cs, tid);
  const T *in = reinterpret_cast<const T *>(A.in) + (size_t)job * A.in_stride;
  const bool init = (A.flags & F_LAMBDA_INIT) != 0;
  const T *lsrc = init ? reinterpret_cast<const T *>(A.table) + (size_t)job * A.table_stride
                       : reinterpret_cast<const T *>(A.lam_in) + (size_t)job * A.lam_stride;
  T *out = reinterpret_cast<T *>(A.out) + (size_t)job * A.out_stride;
  double *part = A.part + (size_t)job * A.part_stride;
  const uint32_t gm = A.gate_mask;

  // copy one array of tile bx into shared tile dst (one commit group); warp w
  // copies tile amplitudes [1024 w, 1024 w + 1024), the ones its rounds L and M read.
  // Chunk m of the thread is tile index i0 + 32 CH m; the bits of m sit above
  // i0's, and a tile index maps bitwise to its global offset, so the offset is
  // go(i0) plus one per-pass weight per set bit of m (computed once here).
  constexpr int IB = (CH == 4) ? 7 : 6;  // log2(32 CH): tile bit of m's bit 0
  constexpr int MB = (CPT == 8) ? 3 : 4;  // bits of m
  static_assert((1 << MB) == CPT && (32 * CH) == (1 << IB), "chunk layout");
  const uint32_t i0 = (uint32_t)(lane * CH + 1024 * w);
  const uint32_t g0 = FULL ? i0 : tile_goff(i0, A);
  uint32_t wm[MB];
#pragma unroll
  for (int j = 0; j < MB; ++j) {
    const int b = IB + j;
    wm[j] = FULL ? (1u << b) : gbit(b, A);
  }
  auto issue = [&](const T *src, uint32_t base, T *dst) {
    const T *gb = src + (base + g0);
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
      uint32_t off = 0;
#pragma unroll
      for (int j = 0; j < MB; ++j)
        if ((m >> j) & 1) off += wm[j];
      cp_async16(dst + swz<T>((int)(i0 + (uint32_t)(32 * CH * m))), gb + off);
    }
    cp_async_commit();
  };

  uint32_t bx = blockIdx.x;
  int par = 0;              // tile parity (gred / ered)
  T *const sp = buf;
  T *const sl = buf + TILE;
  // this tile's index and global base; a thread's global offsets relative to
  // the base are the same for every tile
  uint32_t t = bx < tiles ? tile_of_block(bx, tiles, pair) : 0u;
  uint32_t base = tile_base(t, A, TB);
  if (bx < tiles) {
    issue(in, base, sp);
    issue(lsrc, base, sl);
  }
  GIdx<TB, FULL> grel;
  grel.init(0u, A, lane, w, tid);
  __syncthreads();  // gate coefficients visible
  T2 pthrL;
  if constexpr (CPLX) pthrL = zt.thread_phase_L(lane, w);
  for (; bx < tiles; bx += gridDim.x) {
    const uint32_t nbx = bx + gridDim.x;
    const bool more = nbx < tiles;
    const uint32_t nt = more ? tile_of_block(nbx, tiles, pair) : 0u;
    const uint32_t nbase = more ? tile_base(nt, A, TB) : 0u;
    cp_async_wait<0>();  // this tile's psi and lambda have landed (this warp's part)
    __syncwarp();
    GIdx<TB, FULL> gi = grel;
    gi.baseL += base;
    gi.baseH += base;

    Reg32<T> psi, lam;
    // round L (from shared)
    lds_L(sp, sb, psi);
    lds_L(sl, sb, lam);
    if (init) {
      T eacc = T(0);
#pragma unroll
      for (int k = 0; k < ROUND; ++k) {
        const T p = psi.get(k);
        const T l = lam.get(k) * p;  // the buffer holds the table: lambda = E(x) psi
        lam.set(k, l);
        eacc += p * l;
      }
      if (!CPLX) sts_L(sl, sb, lam);
      eacc = warp_sum(eacc);
      if (lane == 0) ered[par][w] = (double)eacc;
    }
    if constexpr (CPLX) {
      // RZ(-theta) of every qubit of the pass on psi and lambda: both then sit
      // between the pass's RY and RZ gates, where the RY gradients are the plain
      // Im<lam|Y_q|psi> (the other RY gates commute with Y_q) and from where
      // lambda continues through RY(-theta).  The RZ gradients Im<lam|Z_q|psi>
      // are the same on either side of the common phase.
#pragma unroll
      for (int m = 0; m < ROUND / 2; ++m) {
        const T2 ph = cconj(cmul(pthrL, zt.pregL[m]));
        psi.set_pair(m, cmul(psi.pair(m), ph));
        lam.set_pair(m, cmul(lam.pair(m), ph));
      }
      sts_L(sp, sb, psi);
      sts_L(sl, sb, lam);
    }
    round_grads<4, 1, false>(psi, lam, gm, 6, gred[par][w], lane);
    if constexpr (CPLX) rz_grads_L(psi, lam, gm, gredz[par][w], lane, w);
    if (init || CPLX) __syncwarp();  // the rewritten lambda (and psi) are in shared before round M reads them
    // round M (gradients only)
    if (gm & 0x1Fu) {
      lds_M(sp, tid, psi);
      lds_M(sl, tid, lam);
      round_grads<5, 0, false>(psi, lam, gm, 0, gred[par][w], lane);
    }
    // round H: gradients, then RY(-theta) on lambda.  Its layout crosses warps.
    __syncthreads();
    lds_H<TB>(sp, sb, psi);
    lds_H<TB>(sl, sb, lam);
    round_grads<H, 2, true>(psi, lam, gm, 10, gred[par][w], lane);
    round_gates<H, false, true, 2>(lam, gt, gm, 10, true);
    round_gates<1, false, true, 1>(lam, gt, gm, 5, true);
    sts_H<TB>(sl, sb, lam);  // the places this thread read
    __syncthreads();  // psi fully read; lambda in round-H order written
    if (more) issue(in, nbase, sp);  // next psi into the psi buffer
    if (gm & 0x1Fu) {
      lds_M(sl, tid, lam);
      round_gates<5, false>(lam, gt, gm, 0, true);
      sts_M(sl, tid, lam);
      __syncwarp();  // M -> L stays inside the warp's 1024 amplitudes
    }
    lds_L(sl, sb, lam);
    __syncwarp();  // every lane has read its lambda: only this warp reads its part
    if (more) issue(lsrc, nbase, sl);  // next lambda into this warp's part of the lambda buffer
    round_gates<4, false, true, 1>(lam, gt, gm, 6, true);
    // (the short closed forms compute each x from y: measured faster here than
    // the XOR walk, which the other forms take).  The complex path's layer 0
    // (FULL, no entangler) stores plainly or not at all.
    if (FULL && A.store_mode != ST_SCATTER) {
      if (A.store_mode == ST_PLAIN)
        for_L(gi, [&](int m, uint32_t y) { *reinterpret_cast<T2 *>(out + y) = lam.pair(m); });
    } else if (!FULL || (A.em.form <= EF_PREFIX && A.em.sh == 0)) {
      const EntMap em = A.em;
      for_L(gi, [&](int m, uint32_t y) {
        const T2 v = lam.pair(m);
        if constexpr (FULL) {
          uint32_t x;
          if (em.form == EF_PREFIX) {
            x = ent_inv_f<EF_PREFIX>(y, nmask, em, A.n);
          } else {
            x = ent_inv_f<EF_DIFF>(y, nmask, em, A.n);
            if (em.form == EF_WRAP_DIFF) x ^= (x >> (A.n - 1)) & 1u;
          }
          out[x] = v.x;
          out[x ^ d1] = v.y;
        } else {
          *reinterpret_cast<T2 *>(out + y) = v;
        }
      });
    } else if constexpr (FULL) {
      for_L_ent(gi, nmask, A.em, A.n, [&](int m, uint32_t x) {
        const T2 v = lam.pair(m);
        if constexpr (CPLX) {
          *reinterpret_cast<T2 *>(out + x) = v;  // the map keeps the channel bit
        } else {
          out[x] = v.x;
          out[x ^ d1] = v.y;
        }
      });
    }
    // gred / ered of this tile were written before the round-H barriers
    if (tid < TB && ((gm >> tid) & 1u)) {
      double g = 0.0;
#pragma unroll
      for (int ww = 0; ww < NW; ++ww) g += (double)gred[par][ww][tid];
      part[(size_t)tid * tiles + t] = g;
      if constexpr (CPLX) {  // RZ rows follow the TB RY rows
        double gz = 0.0;
#pragma unroll
        for (int ww = 0; ww < NW; ++ww) gz += (double)gredz[par][ww][tid];
        part[(size_t)(TB + tid) * tiles + t] = gz;
      }
    }
    if ((A.flags & F_ENERGY) && tid == 0) {
      double e = 0.0;
#pragma unroll
      for (int ww = 0; ww < NW; ++ww) e += ered[par][ww];
      A.epart[(size_t)job * A.part_stride + t] = e;
    }
    // gred / ered of this parity are rewritten two tiles later, after the next
    // tile's round-H barrier, which warp 0 passes only after the sums above.
    par ^= 1;
    t = nt;
    base = nbase;
  }
  cp_async_wait<0>();
}

// One tile of a backward pass with the loads straight into registers (no
// prefetch); used by the persistent batch kernel, where the next work item is
// a tile of any step.  Same rounds and results as k_bwd.
template <typename T, int TB, bool FULL>
__device__ __forceinline__ void bwd_tile(const PassArgs &A, int job, uint32_t tb_idx) {
  using T2 = typename V2<T>::type;
  constexpr int NT = 1 << (TB - 5);
  constexpr int NW = NT / 32;
  constexpr int H = TB - 10;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sp = reinterpret_cast<T *>(smem_raw);
  T *sl = sp + (1 << TB);
  __shared__ GateTab<T2> gt;
  __shared__ T gred[NW][16];
  __shared__ double ered[NW];

  if (A.minlayer != nullptr && !(A.flags & F_ENERGY) && A.layer < A.minlayer[A.job0 + job]) return;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const SBase sb = sbase<TB, T>(tid);
  const uint32_t t = tile_of_block(tb_idx, (uint32_t)A.tiles, A.pair_mask);
  const uint32_t tbase = tile_base(t, A, TB);
  const uint32_t nmask = (1u << A.n) - 1;
  const uint32_t d1 = ent_inv(1u, nmask, A.em, A.n);  // the pair (y, y + 1) maps to (x, x ^ d1)
  const T2 *cs = reinterpret_cast<const T2 *>(A.cs) + (size_t)(A.job0 + job) * A.P;
  load_gate_coeffs(A, cs, gt.cs, tid);
  if (sizeof(T) == 4) gt.pack(tid);
  const T *in = reinterpret_cast<const T *>(A.in) + (size_t)job * A.in_stride;
  const T *lin = reinterpret_cast<const T *>(A.lam_in) + (size_t)job * A.lam_stride;
  const T *table = reinterpret_cast<const T *>(A.table) + (size_t)job * A.table_stride;
  T *out = reinterpret_cast<T *>(A.out) + (size_t)job * A.out_stride;
  const uint32_t gm = A.gate_mask;
  const bool init = (A.flags & F_LAMBDA_INIT) != 0;
  GIdx<TB, FULL> gi;
  gi.init(tbase, A, lane, w, tid);

  // round L loads go out before the barrier that publishes the gate
  // coefficients (they do not depend on them); the shared partials and tiles
  // are written after it, once the previous item's epilogue has read them
  Reg32<T> psi, lam;
  T eacc = T(0);
  for_L(gi, [&](int m, uint32_t y) {
    const T2 p = __ldcg(reinterpret_cast<const T2 *>(in + y));
    T2 l;
    if (init) {
      l.x = table[y] * p.x;
      l.y = table[y + 1] * p.y;
    } else {
      l = __ldcg(reinterpret_cast<const T2 *>(lin + y));
    }
    psi.set_pair(m, p);
    lam.set_pair(m, l);
    eacc += p.x * l.x + p.y * l.y;
  });
  __syncthreads();
  round_grads<4, 1>(psi, lam, gm, 6, gred[w], lane);
  sts_L(sp, sb, psi);
  sts_L(sl, sb, lam);
  if (A.flags & F_ENERGY) {
    eacc = warp_sum(eacc);
    if (lane == 0) ered[w] = (double)eacc;
  }
  __syncwarp();  // L -> M stays inside the warp's 1024 amplitudes
  if (gm & 0x1Fu) {
    lds_M(sp, tid, psi);
    lds_M(sl, tid, lam);
    round_grads<5>(psi, lam, gm, 0, gred[w], lane);
  }
  __syncthreads();  // round H reads across warps, after every warp's round M
  lds_H<TB>(sp, sb, psi);
  lds_H<TB>(sl, sb, lam);
  round_grads<H, 2, true>(psi, lam, gm, 10, gred[w], lane);
  round_gates<H, false, true, 2>(lam, gt, gm, 10, true);
  round_gates<1, false, true, 1>(lam, gt, gm, 5, true);
  sts_H<TB>(sl, sb, lam);  // the places this thread read
  __syncthreads();
  if (gm & 0x1Fu) {
    lds_M(sl, tid, lam);
    round_gates<5, false>(lam, gt, gm, 0, true);
    sts_M(sl, tid, lam);
    __syncwarp();  // M -> L stays inside the warp's 1024 amplitudes
  }
  lds_L(sl, sb, lam);
  round_gates<4, false, true, 1>(lam, gt, gm, 6, true);
  if constexpr (FULL) {
    for_L_ent(gi, nmask, A.em, A.n, [&](int m, uint32_t x) {
      const T2 v = lam.pair(m);
      out[x] = v.x;
      out[x ^ d1] = v.y;
    });
  } else {
    for_L(gi, [&](int m, uint32_t y) { *reinterpret_cast<T2 *>(out + y) = lam.pair(m); });
  }
  __syncthreads();
  double *part = A.part + (size_t)job * A.part_stride;
  if (tid < TB && ((gm >> tid) & 1u)) {
    double g = 0.0;
#pragma unroll
    for (int ww = 0; ww < NW; ++ww) g += (double)gred[ww][tid];
    part[(size_t)tid * A.tiles + t] = g;
  }
  if ((A.flags & F_ENERGY) && tid == 0) {
    double e = 0.0;
#pragma unroll
    for (int ww = 0; ww < NW; ++ww) e += ered[ww];
    A.epart[(size_t)job * A.part_stride + t] = e;
  }
  __syncthreads();
}

// ------------------------------------------------ layer-0 gradient pass --
// g_{0,q} = sum_x lambda_0[x] prod_{q' != q} f_q'(x_q') d_q(x_q) with
// f(0) = cos(t/2), f(1) = sin(t/2), d(0) = -sin(t/2), d(1) = cos(t/2): the
// adjoint formula evaluated against the layer-0 product state.  The tile is
// global bits [0, TB); the product over the register bits 5..9 is tabulated.
template <typename T, int TB>
__device__ __forceinline__ void grad_l0_tile(const PassArgs &A, int job, uint32_t t) {
  using T2 = typename V2<T>::type;
  constexpr int NT = 1 << (TB - 5);
  constexpr int NW = NT / 32;
  constexpr int NV = 11;  // per-thread values reduced over the warp
  __shared__ T2 l0cs[32];
  __shared__ T RF[ROUND], RD[5][ROUND];
  __shared__ double wv[NW][NV];
  __shared__ double ered[NW];
  __shared__ double fhi_d[32];
  __shared__ double fhi_all;

  if (A.minlayer != nullptr && !(A.flags & F_ENERGY) && A.minlayer[A.job0 + job] > 0) return;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int n = A.n;
  const T2 *cs = reinterpret_cast<const T2 *>(A.cs) + (size_t)(A.job0 + job) * A.P;
  if (tid < n) l0cs[tid] = cs[tid];
  __syncthreads();
  if (tid < ROUND) {
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
  const T *lin = reinterpret_cast<const T *>(A.lam_in) + (size_t)job * A.lam_stride;
  const T *table = reinterpret_cast<const T *>(A.table) + (size_t)job * A.table_stride;
  const uint32_t tbase = t << TB;
  const T fhi_t = (T)fhi_all;
  T S = T(0), Sj[5] = {T(0), T(0), T(0), T(0), T(0)};
  T eacc = T(0);
#pragma unroll
  for (int k = 0; k < ROUND; ++k) {
    const uint32_t x = tbase + lane + 32 * k + 1024 * w;
    T lam;
    if (init) {
      const T psi0 = lane_f * RF[k] * warp_f * fhi_t;
      lam = table[x] * psi0;
      eacc += psi0 * lam;
    } else {
      lam = __ldcg(lin + x);
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

  double *part = A.part + (size_t)job * A.part_stride;
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
    part[(size_t)q * A.tiles + t] = g;
  }
  if (init && tid == 0) {
    double e = 0.0;
    for (int ww = 0; ww < NW; ++ww) e += ered[ww];
    A.epart[(size_t)job * A.part_stride + t] = e;
  }
  __syncthreads();
}

// ----------------------------------------- lambda = H psi with X-mask groups --
// lambda[x] = E(x) psi[x] + sum_groups D_m(x ^ m) psi[x ^ m] with
// D_m(u) = sum_{k in group} c_k (-1)^popcount(u & z_k) (c_k carries the i^#Y sign).
//
// A CTA owns the output tile t (2^TB amplitudes, 32 per thread in registers:
// FP32 as 16 packed pairs of neighbouring elements, see xy_group_pk).
// The groups come sorted by X-mask m, so groups whose mask agrees above the
// tile bits (the same high part h = m >> TB) form consecutive runs; a run needs
// one partner tile, psi over tile t ^ h, which is streamed into shared memory
// with cp.async, the next run's partner landing in the other buffer while this
// run's groups are applied.  For element e of the tile (u = x ^ m has tile part
// e ^ m_lo), the sign (-1)^popcount(u & z) splits into a part constant over the
// CTA (the tile index bits of u), one constant per thread (its thread bits of
// e ^ m_lo) and one that depends only on the register slot k, read from a
// 32-bit mask per term built once per CTA: no population count per element.
// Bytes: psi and the table of tile t, one partner tile per run, lambda written.
// One X-mask group applied to a thread's 32 elements (FP64): element k (tile
// index e = k NT + tid) gains D(u) psi[u] with u's tile part k NT ^ tm read from
// the partner tile; D(u) = sum_j c[j] (-1)^(bit k of km[j]), the signs of u's
// other bits already folded into c[j].  NTERM terms (unused ones have c = 0).
template <typename T, int TB, int NTERM>
__device__ __forceinline__ void xy_group(T (&acc)[ROUND], const T *buf, uint32_t tm, const T (&c)[4],
                                         const uint32_t (&km)[4]) {
  constexpr int NT = 1 << (TB - 5);
#pragma unroll
  for (int k = 0; k < ROUND; ++k) {
    T d = flip_sign(c[0], (km[0] >> k) & 1u);
#pragma unroll
    for (int j = 1; j < NTERM; ++j) d += flip_sign(c[j], (km[j] >> k) & 1u);
    acc[k] += d * buf[((uint32_t)(k * NT)) ^ tm];
  }
}

// The FP32 form: a thread owns 16 pairs of neighbouring elements, pair j holding
// tile indices e = j 2^(TB-4) + 2 tid and e + 1; their partners e ^ m_lo and
// e ^ m_lo ^ 1 share one 8-byte word (in swapped order when bit 0 of m_lo is
// set), and a term's two signs differ by bit 0 of z, so each pair takes one
// 8-byte shared load and packed f32x2 arithmetic.  c2[t] holds the term's pair
// of signed coefficients, km[t] bit j the sign pair j's slot bits add.
template <int TB, int NTERM, bool SWAP>
__device__ __forceinline__ void xy_group_pk(unsigned long long (&acc)[ROUND / 2], const float *buf, uint32_t tm,
                                            const unsigned long long (&c2)[4], const uint32_t (&km)[4]) {
  const float2 *b2 = reinterpret_cast<const float2 *>(buf);
#pragma unroll
  for (int j = 0; j < ROUND / 2; ++j) {
    const float2 p = b2[(((uint32_t)j << (TB - 4)) ^ tm) >> 1];
    const unsigned long long p2 = SWAP ? pk(p.y, p.x) : pk(p.x, p.y);
    auto signed_c = [&](int t) {
      const uint32_t sb = (km[t] << (31 - j)) & 0x80000000u;
      return c2[t] ^ (((unsigned long long)sb << 32) | sb);
    };
    unsigned long long d2 = signed_c(0);
#pragma unroll
    for (int t = 1; t < NTERM; ++t) d2 = add2(d2, signed_c(t));
    acc[j] = fma2(d2, p2, acc[j]);
  }
}

template <typename T, int TB>
__global__ void __launch_bounds__(1 << (TB - 5)) k_lambda_xy(const PassArgs A) {
  constexpr int NT = 1 << (TB - 5);
  constexpr int NW = NT / 32;
  constexpr uint32_t LOW = (1u << TB) - 1u;
  constexpr bool PAIRS = sizeof(T) == 4;  // FP32: packed pairs of neighbouring elements
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nterm = A.ngroups > 0 ? A.gstart[A.ngroups] - A.gstart[0] : 0;
  const XyLayout lay = xy_layout(A.ngroups, nterm, (int)sizeof(T));
  uint32_t *sgm = reinterpret_cast<uint32_t *>(smem_raw + lay.gm);
  int *sgs = reinterpret_cast<int *>(smem_raw + lay.gs);
  uint32_t *stz = reinterpret_cast<uint32_t *>(smem_raw + lay.tz);
  T *stc = reinterpret_cast<T *>(smem_raw + lay.tc);
  int *srun = reinterpret_cast<int *>(smem_raw + lay.runs);
  uint32_t *skm = reinterpret_cast<uint32_t *>(smem_raw + lay.km);
  T *sbuf = reinterpret_cast<T *>(smem_raw + lay.buf);
  __shared__ double ered[NW];
  __shared__ int s_nruns;
  const int job = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t t = blockIdx.x;
  const int t0 = A.ngroups > 0 ? A.gstart[0] : 0;
  for (int i = tid; i < A.ngroups; i += NT) sgm[i] = A.gmask[i];
  if (A.ngroups > 0)
    for (int i = tid; i <= A.ngroups; i += NT) sgs[i] = A.gstart[i] - t0;
  for (int i = tid; i < nterm; i += NT) {
    const uint32_t z = A.tz[t0 + i];
    stz[i] = z;
    stc[i] = reinterpret_cast<const T *>(A.tc)[t0 + i];
    // bit k: the parity of z over the slot bits of register slot k (FP64: slot
    // k is tile bits TB-5.. of k NT; FP32: pair k is tile bits TB-4.. of k 2^(TB-4))
    const int sbits = PAIRS ? 4 : 5;
    const uint32_t zk = (z >> (TB - sbits)) & ((1u << sbits) - 1u);
    uint32_t km = 0;
    for (int k = 0; k < (1 << sbits); ++k) km |= (uint32_t)(__popc((uint32_t)k & zk) & 1) << k;
    skm[i] = km;
  }
  __syncthreads();
  if (tid == 0) {  // runs of equal high part (groups arrive sorted by mask)
    int nr = 0;
    for (int g = 0; g < A.ngroups; ++g)
      if (g == 0 || (sgm[g] >> TB) != (sgm[g - 1] >> TB)) srun[nr++] = g;
    srun[nr] = A.ngroups;
    s_nruns = nr;
  }
  const T *in = reinterpret_cast<const T *>(A.in) + (size_t)job * A.in_stride;
  const T *lin = reinterpret_cast<const T *>(A.lam_in) + (size_t)job * A.lam_stride;
  const T *table = reinterpret_cast<const T *>(A.table) + (size_t)job * A.table_stride;
  T *out = reinterpret_cast<T *>(A.out) + (size_t)job * A.out_stride;
  const uint32_t tbase = t << TB;
  // the thread's elements: FP64 e = k NT + tid; FP32 pairs (j 2^(TB-4) + 2 tid, + 1)
  const uint32_t tpart = PAIRS ? (uint32_t)tid << 1 : (uint32_t)tid;
  T acc[PAIRS ? 1 : ROUND];
  unsigned long long acc2[PAIRS ? ROUND / 2 : 1];
  if constexpr (PAIRS) {
#pragma unroll
    for (int j = 0; j < ROUND / 2; ++j) {
      const uint32_t x = tbase + ((uint32_t)j << (TB - 4)) + tpart;
      float2 v;
      if (A.flags & F_ACCUM) {
        v = *reinterpret_cast<const float2 *>(lin + x);
      } else {
        const float2 p = *reinterpret_cast<const float2 *>(in + x);
        const float2 e = *reinterpret_cast<const float2 *>(table + x);
        v = make_float2(e.x * p.x, e.y * p.y);
      }
      acc2[j] = pk(v);
    }
  } else {
#pragma unroll
    for (int k = 0; k < ROUND; ++k) {
      const uint32_t x = tbase + (uint32_t)(k * NT) + tpart;
      acc[k] = (A.flags & F_ACCUM) ? lin[x] : table[x] * in[x];
    }
  }
  __syncthreads();
  const int nruns = s_nruns;
  constexpr int CHUNKS = (int)((sizeof(T) << TB) / 16);  // 16-byte pieces of one tile
  auto load_partner = [&](int r, int b) {
    const uint32_t pt = t ^ (sgm[srun[r]] >> TB);
    const char *src = reinterpret_cast<const char *>(in + ((size_t)pt << TB));
    char *dst = reinterpret_cast<char *>(sbuf + ((size_t)b << TB));
    for (int i = tid; i < CHUNKS; i += NT) cp_async16(dst + 16 * i, src + 16 * (size_t)i);
    cp_async_commit();
  };
  if (nruns > 0) load_partner(0, 0);
  for (int r = 0; r < nruns; ++r) {
    if (r + 1 < nruns) {
      load_partner(r + 1, (r + 1) & 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const T *buf = sbuf + ((size_t)(r & 1) << TB);
    const uint32_t hi_bits = (t ^ (sgm[srun[r]] >> TB)) << TB;  // tile-index bits of u
    for (int g = srun[r]; g < srun[r + 1]; ++g) {
      const uint32_t mlo = sgm[g] & LOW;
      const uint32_t tm = tpart ^ mlo;  // the partner of the thread's (first) element, less the slot bits
      const int j0 = sgs[g], nt = sgs[g + 1] - j0;
      if constexpr (PAIRS) {
        // per term: the pair of coefficients with the signs of every bit of u but
        // the slot bits folded in (the pair's second element adds bit 0 of z)
        auto load_terms = [&](int jb, unsigned long long (&c2)[4], uint32_t (&km)[4]) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (jb + j < j0 + nt) {
              const uint32_t z = stz[jb + j];
              const float c0 = flip_sign(stc[jb + j], __popc(z & (hi_bits | tm)) & 1);
              c2[j] = pk(c0, flip_sign(c0, z & 1u));
              km[j] = skm[jb + j];
            } else {
              c2[j] = 0ull;
              km[j] = 0;
            }
          }
        };
        unsigned long long c2[4];
        uint32_t km[4];
        const bool swap = (mlo & 1u) != 0;
        const float *f = reinterpret_cast<const float *>(buf);
        for (int jb = j0; jb < j0 + nt; jb += 4) {
          load_terms(jb, c2, km);
          const int left = j0 + nt - jb;
          if (left == 1) {
            swap ? xy_group_pk<TB, 1, true>(acc2, f, tm, c2, km) : xy_group_pk<TB, 1, false>(acc2, f, tm, c2, km);
          } else if (left == 2) {
            swap ? xy_group_pk<TB, 2, true>(acc2, f, tm, c2, km) : xy_group_pk<TB, 2, false>(acc2, f, tm, c2, km);
          } else {
            swap ? xy_group_pk<TB, 4, true>(acc2, f, tm, c2, km) : xy_group_pk<TB, 4, false>(acc2, f, tm, c2, km);
          }
        }
      } else {
        // per term: its coefficient with the sign of every bit of u but the slot bits
        // folded in, and its slot mask (bit k: the sign the slot bits of k add)
        T c[4];
        uint32_t km[4];
        for (int jb = j0; jb < j0 + nt; jb += 4) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (jb + j < j0 + nt) {
              c[j] = flip_sign(stc[jb + j], __popc(stz[jb + j] & (hi_bits | tm)) & 1);
              km[j] = skm[jb + j];
            } else {
              c[j] = T(0);
              km[j] = 0;
            }
          }
          const int left = j0 + nt - jb;
          if (left == 1)
            xy_group<T, TB, 1>(acc, buf, tm, c, km);
          else if (left == 2)
            xy_group<T, TB, 2>(acc, buf, tm, c, km);
          else
            xy_group<T, TB, 4>(acc, buf, tm, c, km);
        }
      }
    }
    __syncthreads();  // every thread is done with this buffer before it is refilled
  }
  T eacc = T(0);
  if constexpr (PAIRS) {
#pragma unroll
    for (int j = 0; j < ROUND / 2; ++j) {
      const uint32_t x = tbase + ((uint32_t)j << (TB - 4)) + tpart;
      const float2 v = upk(acc2[j]);
      if (A.flags & F_WRITE_LAMBDA) *reinterpret_cast<float2 *>(out + x) = v;
      const float2 p = *reinterpret_cast<const float2 *>(in + x);
      eacc += p.x * v.x + p.y * v.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < ROUND; ++k) {
      const uint32_t x = tbase + (uint32_t)(k * NT) + tpart;
      if (A.flags & F_WRITE_LAMBDA) out[x] = acc[k];
      eacc += in[x] * acc[k];
    }
  }
  if (A.flags & F_ENERGY) {
    eacc = warp_sum(eacc);
    if (lane == 0) ered[w] = (double)eacc;
    __syncthreads();
    if (tid == 0) {
      double e = 0.0;
      for (int ww = 0; ww < NW; ++ww) e += ered[ww];
      A.epart[(size_t)job * A.part_stride + t] = e;
    }
  }
}

// ------------------------------------------------------------- launcher --
inline int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
  }
  return n;
}

template <typename K>
static cudaError_t launch_k(K k, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const PassArgs &A) {
  if (smem > 0) {  // dynamic + static shared memory may cross the 48 KiB default
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k<<<grid, block, smem, s>>>(A);
  return cudaGetLastError();
}

// A persistent kernel: as many CTAs as are resident on the device at once
// (the occupancy calculator's count per SM, cached per kernel), split over the
// jobs, and never more than the tiles of one job.
static cudaError_t launch_persistent(void (*k)(const PassArgs), int jobs, long long tiles, dim3 block, size_t smem,
                                     cudaStream_t s, const PassArgs &A) {
  static std::mutex mu;
  static std::unordered_map<const void *, int> per_sm_of;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = per_sm_of.find((const void *)k);
    if (it != per_sm_of.end()) {
      per_sm = it->second;
    } else {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, (int)block.x, smem);
      if (e != cudaSuccess) return e;
      if (per_sm < 1) return cudaErrorInvalidConfiguration;
      per_sm_of[(const void *)k] = per_sm;
    }
  }
  long long ctas = (long long)num_sms() * per_sm / jobs;
  if (ctas < 1) ctas = 1;
  if (ctas > tiles) ctas = tiles;
  k<<<dim3((unsigned)ctas, (unsigned)jobs), block, smem, s>>>(A);
  return cudaGetLastError();
}

template <typename T, int TB>
cudaError_t launch_tb(const PassArgs &A, int jobs, int nterm, cudaStream_t s) {
  const dim3 grid((unsigned)A.tiles, (unsigned)jobs);
  const dim3 block(1 << (TB - 5));
  const size_t tile = sizeof(T) << TB;
  const bool full = A.c >= TB;
  switch (A.kind) {
    case K_FWD:
      if (A.flags & F_COMPLEX) {
        if (!full) {
          if (A.load_mode != LD_PLAIN) return cudaErrorInvalidValue;
          return launch_k(k_fwd<T, TB, false, LD_PLAIN, false, true>, grid, block, tile, s, A);
        }
        switch (A.load_mode) {
          case LD_PLAIN: return launch_k(k_fwd<T, TB, true, LD_PLAIN, false, true>, grid, block, tile, s, A);
          case LD_GATHER: return launch_k(k_fwd<T, TB, true, LD_GATHER, false, true>, grid, block, tile, s, A);
          case LD_ZERO: return launch_k(k_fwd<T, TB, true, LD_ZERO, false, true>, grid, block, tile, s, A);
          default: return cudaErrorInvalidValue;
        }
      }
      if (!full) {
        if (A.load_mode != LD_PLAIN) return cudaErrorInvalidValue;
        return launch_k(k_fwd<T, TB, false, LD_PLAIN, false>, grid, block, tile, s, A);
      }
      switch (A.load_mode) {
        case LD_PLAIN: return launch_k(k_fwd<T, TB, true, LD_PLAIN, false>, grid, block, tile, s, A);
        case LD_GATHER: return launch_k(k_fwd<T, TB, true, LD_GATHER, false>, grid, block, tile, s, A);
        case LD_L0_GATHER: return launch_k(k_fwd<T, TB, true, LD_L0_GATHER, false>, grid, block, tile, s, A);
        case LD_L0: return launch_k(k_fwd<T, TB, true, LD_L0, false>, grid, block, tile, s, A);
        default: return cudaErrorInvalidValue;
      }
    case K_WHT:
      if (full) return launch_k(k_fwd<T, TB, true, LD_PLAIN, true>, grid, block, tile, s, A);
      return launch_k(k_fwd<T, TB, false, LD_PLAIN, true>, grid, block, tile, s, A);
    case K_BWD: {
      // the first pass of a layer (layout FULL) writes lambda through the inverse CX
      // chain; the complex path's layer 0 (no entangler) stores plainly or not at all
      const bool cplx = (A.flags & F_COMPLEX) != 0;
      if (!full && A.store_mode != ST_PLAIN) return cudaErrorInvalidValue;
      if (full && !cplx && A.store_mode != ST_SCATTER) return cudaErrorInvalidValue;
      void (*k)(const PassArgs) = cplx ? (full ? k_bwd<T, TB, true, true> : k_bwd<T, TB, false, true>)
                                       : (full ? k_bwd<T, TB, true> : k_bwd<T, TB, false>);
      return launch_persistent(k, jobs, A.tiles, block, 2 * tile, s, A);
    }
    case K_LAMBDA_XY: {
      const size_t smem = xy_layout(A.ngroups, nterm, (int)sizeof(T), TB).total;
      if (smem > 200 * 1024) return cudaErrorInvalidValue;
      return launch_k(k_lambda_xy<T, TB>, grid, block, smem, s, A);
    }
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace gvqe
