// gvqe_mps.cu -- the leading layers of the RY + CX ansatz in closed form.
//
// The forward state after layer 0 is the product state psi_0(x) = prod_q f_q(x_q),
// f_q(0) = cos(t_q/2), f_q(1) = sin(t_q/2) (Eq. 7 applied to |0>).  Layer k >= 1
// maps it on as (Section IV-B: entangler, then one RY per qubit)
//
//   psi_k(y) = sum_u R_k(y, u) psi_{k-1}(A^-1 u),   R_k(y, u) = prod_q RY_{k,q}(y_q, u_q),
//
// with A the entangler's map of basis indices (y = A x).  For the linear chain,
// x = u ^ (u << 1), bit q of A^-1 u is u_q ^ u_{q-1}; for full and reverse
// linear it is the running parity p_q = u_0 ^ ... ^ u_q.  Either way every
// factor ties qubit q only to qubit q - 1, so summing out the intermediate
// indices qubit by qubit leaves
//
//   psi_r(y) = e_0^T A_0[y_0] A_1[y_1] ... A_{n-1}[y_{n-1}] 1
//
// with D x D site matrices, D = 2^r: the bond between qubits q - 1 and q holds,
// for every layer k <= r, the bit u^k_{q-1} (linear) or the parity p^k_{q-1}
// (prefix); bit k - 1 of a bond index is layer k's.  Site q's entry for left
// bond a and right bond b is
//
//   linear:  f_q(b^1 ^ a^1) * prod_{k<r} RY_{k,q}(b^{k+1} ^ a^{k+1}, b^k) * RY'_{r,q}(y_q, b^r)
//   prefix:  f_q(b^1)       * prod_{k<r} RY_{k,q}(b^{k+1}, b^k ^ a^k)     * RY'_{r,q}(y_q, b^r ^ a^r)
//
// (a = 0 at q = 0; the right end sums over b), where RY' is layer r's rotation
// on the qubits the stage has applied and the identity on the others: the
// stored states between the passes of layer r are such stages.  The result is
// the state the gate passes compute, up to rounding.
//
// k_mps_tab contracts the site matrices (from the same FP32 cos/sin values the
// gate passes use, in FP64) into four tables, rounded once to FP32: the row
// vector of qubits [0, 7) per pattern, the matrices of [7, 13) and [13, 13 + h1)
// and the column vector of [13 + h1, n).  k_mps_write then produces each
// 2^13-amplitude chunk as r = M_h1 v_h2 (one vector per chunk), m = M_mid r (one
// per pattern of qubits 7..12) and psi(y) = L(y_0..6) . m(y_7..12): D FMAs per
// amplitude and one 16-byte store per four, a write-only stream.
#include "gvqe_tile.cuh"

namespace gvqe {

int num_sms_cached();

namespace {

__device__ __forceinline__ double ry_entry(float2 g, int out, int in) {
  return out == in ? (double)g.x : (out ? (double)g.y : -(double)g.y);
}

// Site matrix entry A_q[y](a, b) of the stage (layer r, layer r's rotated qubits rot).
template <int FORM>
__device__ double site_entry(const float2 *cs, int pstride, int q, int y, int a, int b, int r, bool rot) {
  if (q == 0 && a != 0) return 0.0;  // the left end's bond is 0
  auto bit = [](int v, int k) { return (v >> (k - 1)) & 1; };
  const float2 f = cs[q];
  const int x0 = (FORM == EF_PREFIX) ? bit(b, 1) : (bit(b, 1) ^ bit(a, 1));
  double v = x0 ? (double)f.y : (double)f.x;
  for (int k = 1; k <= r; ++k) {
    int out, in;
    if (FORM == EF_PREFIX) {
      out = (k < r) ? bit(b, k + 1) : y;
      in = bit(b, k) ^ bit(a, k);
    } else {
      out = (k < r) ? (bit(b, k + 1) ^ bit(a, k + 1)) : y;
      in = bit(b, k);
    }
    if (k == r && !rot) {
      if (out != in) return 0.0;
      continue;
    }
    v *= ry_entry(cs[(size_t)k * pstride + q], out, in);
  }
  return v;
}

// Table sections, in item order: 128 rows of [0, 7), 64 D rows of [7, 13),
// 2^h1 D rows of [13, 13 + h1), 2^h2 columns of [13 + h1, n).
struct MpsItems {
  long long lo, mid, m1, r2, total;
};
__host__ __device__ inline MpsItems mps_items(const MpsDims &d) {
  MpsItems it;
  it.lo = 128;
  it.mid = it.lo + 64LL * d.D;
  it.m1 = it.mid + (1LL << d.h1) * d.D;
  it.r2 = it.m1 + (1LL << d.h2);
  it.total = it.r2;
  return it;
}
constexpr int TAB_NT = 64;

// The qubits a table section's items contract over.
__host__ __device__ inline int mps_q_first(const MpsItems &its, const MpsDims &d, long long i) {
  return i < its.lo ? 0 : (i < its.mid ? 7 : (i < its.m1 ? 13 : 13 + d.h1));
}
__host__ __device__ inline int mps_q_last(const MpsItems &its, const MpsDims &d, int n, long long i) {
  return i < its.lo ? 6 : (i < its.mid ? 12 : (i < its.m1 ? 12 + d.h1 : n - 1));
}
// Site matrices one CTA of k_mps_tab holds: the widest qubit span of any CTA's items.
inline int mps_tab_span(int n, int r) {
  const MpsDims d = mps_dims(n, r);
  const MpsItems its = mps_items(d);
  int span = 1;
  for (long long i0 = 0; i0 < its.total; i0 += TAB_NT) {
    const long long i1 = (i0 + TAB_NT < its.total) ? i0 + TAB_NT : its.total;
    const int w = mps_q_last(its, d, n, i1 - 1) - mps_q_first(its, d, i0) + 1;
    if (w > span) span = w;
  }
  return span;
}

// One CTA of TAB_NT threads takes items [blockIdx.x TAB_NT, +TAB_NT): it
// builds the site matrices of the qubits those items span in shared memory
// (FP64, [q - first qubit][y][a][b]; the host sizes it by mps_tab_span) and
// contracts one table row (or column) per thread.
template <int D, int FORM>
__global__ void __launch_bounds__(TAB_NT) k_mps_tab(const PassArgs A) {
  extern __shared__ double site[];
  constexpr int DD = D * D;
  const int n = A.n, r = A.layer, job = blockIdx.y, tid = threadIdx.x;
  const MpsDims d = mps_dims(n, r);
  const MpsItems its = mps_items(d);
  const float2 *cs = reinterpret_cast<const float2 *>(A.cs) + (size_t)(A.job0 + job) * A.P;
  const long long i0 = (long long)blockIdx.x * TAB_NT;
  const long long i1 = (i0 + TAB_NT < its.total) ? i0 + TAB_NT : its.total;
  const int qa = mps_q_first(its, d, i0), qb = mps_q_last(its, d, n, i1 - 1);
  const int ne = (qb - qa + 1) * 2 * DD;
  for (int e = tid; e < ne; e += TAB_NT) {
    const int b = e % D, a = (e / D) % D, y = (e / DD) & 1, q = qa + e / (2 * DD);
    site[(size_t)(q - qa) * 2 * DD + y * DD + a * D + b] =
        (FORM == EF_PREFIX) ? site_entry<EF_PREFIX>(cs, A.pstride, q, y, a, b, r, (A.gate_mask >> q) & 1u)
                            : site_entry<EF_DIFF>(cs, A.pstride, q, y, a, b, r, (A.gate_mask >> q) & 1u);
  }
  __syncthreads();
  const long long it = i0 + tid;
  if (it >= i1) return;
  float *tab = reinterpret_cast<float *>(A.out) + (size_t)job * A.out_stride;
  auto mat = [&](int q, int y) { return site + (size_t)(q - qa) * 2 * DD + y * DD; };
  double v[D];
  // v <- v A (row vector)
  auto vecmat = [&](const double *M) {
    double t[D];
#pragma unroll
    for (int b = 0; b < D; ++b) {
      double acc = 0.0;
#pragma unroll
      for (int a = 0; a < D; ++a) acc = fma(v[a], M[a * D + b], acc);
      t[b] = acc;
    }
#pragma unroll
    for (int b = 0; b < D; ++b) v[b] = t[b];
  };
  if (it < its.mid) {
    // a row of [0, 7) (from e_0) or of [7, 13) (from e_a)
    const bool lo = it < its.lo;
    const int pat = lo ? (int)it : (int)((it - its.lo) / D);
    const int a0 = lo ? 0 : (int)((it - its.lo) % D);
#pragma unroll
    for (int a = 0; a < D; ++a) v[a] = (a == a0) ? 1.0 : 0.0;
    const int q0 = lo ? 0 : 7, nq = lo ? 7 : 6;
    for (int j = 0; j < nq; ++j) vecmat(mat(q0 + j, (pat >> j) & 1));
    if (lo) {
#pragma unroll
      for (int a = 0; a < D; ++a) tab[d.lo + (long long)a * 128 + pat] = (float)v[a];
    } else {
#pragma unroll
      for (int b = 0; b < D; ++b) tab[d.mid + ((long long)pat * D + a0) * D + b] = (float)v[b];
    }
  } else if (it < its.m1) {
    const long long i = it - its.mid;
    const long long c1 = i / D;
    const int a0 = (int)(i % D);
#pragma unroll
    for (int a = 0; a < D; ++a) v[a] = (a == a0) ? 1.0 : 0.0;
    for (int j = 0; j < d.h1; ++j) vecmat(mat(13 + j, (int)((c1 >> j) & 1)));
#pragma unroll
    for (int b = 0; b < D; ++b) tab[d.m1 + (c1 * D + a0) * D + b] = (float)v[b];
  } else {
    // the column of [13 + h1, n) from the right end (all ones)
    const long long c2 = it - its.m1;
#pragma unroll
    for (int a = 0; a < D; ++a) v[a] = 1.0;
    for (int q = n - 1; q >= 13 + d.h1; --q) {
      const double *M = mat(q, (int)((c2 >> (q - 13 - d.h1)) & 1));
      double t[D];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < D; ++b) acc = fma(M[a * D + b], v[b], acc);
        t[a] = acc;
      }
#pragma unroll
      for (int a = 0; a < D; ++a) v[a] = t[a];
    }
#pragma unroll
    for (int a = 0; a < D; ++a) tab[d.r2 + c2 * D + a] = (float)v[a];
  }
}

constexpr int WR_NT = 256;  // 8 warps; warp w writes the rows w, w + 8, ... of a chunk

// Persistent CTAs walk the 2^13-amplitude chunks.  Lane l of every warp owns
// amplitudes 4l .. 4l + 3 of each 128-amplitude row (qubits 0..6), so its four
// row vectors of [0, 7) stay in registers; a row of the chunk (qubits 7..12)
// is one shared vector m, read as a broadcast.  For D >= 4 the next chunk's
// matrix of [13, 13 + h1) and vector of [13 + h1, n) stream into a second
// shared buffer (cp.async) while this chunk is written, so no chunk waits on
// their loads.
template <int D>
__global__ void __launch_bounds__(WR_NT) k_mps_write(const PassArgs A) {
  extern __shared__ __align__(16) float sM[];  // [64][b][a] (transposed), dynamic (64 KiB at D = 16)
  __shared__ __align__(16) float sm[64 * 2 * D];  // m per row, each value twice: (m_a, m_a) pairs
  __shared__ __align__(16) float sb[2][D * D + D];  // staged [D][D] matrix and [D] vector, by chunk parity
  __shared__ float sr[D];
  constexpr bool STAGE = D >= 4;
  constexpr int NCH = (D * D + D) / 4;  // 16-byte copies per staged chunk
  const int r = (D == 2) ? 1 : (D == 4 ? 2 : (D == 8 ? 3 : 4));
  const MpsDims d = mps_dims(A.n, r);
  const int job = blockIdx.y, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const float *tab = reinterpret_cast<const float *>(A.in) + (size_t)job * A.in_stride;
  float *out = reinterpret_cast<float *>(A.out) + (size_t)job * A.out_stride;
  const long long chunks = A.tiles;
  const long long mask1 = (1LL << d.h1) - 1;
  // one 16-byte piece of chunk c's matrix (pieces 0 .. D D / 4 - 1) or vector
  auto stage = [&](long long c, int buf) {
    if (tid < NCH) {
      const float *src = (tid < D * D / 4) ? tab + d.m1 + (c & mask1) * D * D + 4 * tid
                                           : tab + d.r2 + (c >> d.h1) * D + 4 * (tid - D * D / 4);
      cp_async16(&sb[buf][4 * tid], src);
    }
    cp_async_commit();
  };
  if constexpr (STAGE) stage(blockIdx.x, 0);
  // the matrices of [7, 13) transposed, so that the threads of m = M r (consecutive a)
  // read consecutive words for every b
  for (int i = tid; i < 64 * D * D; i += WR_NT) {
    const int ym = i / (D * D), b = (i / D) % D, a = i % D;
    sM[i] = tab[d.mid + (ym * D + a) * D + b];
  }
  unsigned long long L01[D], L23[D];  // (L[4l], L[4l+1]) and (L[4l+2], L[4l+3]) per bond index
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const float4 l = *reinterpret_cast<const float4 *>(tab + d.lo + a * 128 + 4 * lane);
    L01[a] = pk(l.x, l.y);
    L23[a] = pk(l.z, l.w);
  }
  int par = 0;
  for (long long c = blockIdx.x; c < chunks; c += gridDim.x, par ^= 1) {
    if constexpr (STAGE) cp_async_wait<0>();
    __syncthreads();  // staged data visible; the previous chunk's vectors are read (and sM is loaded)
    if constexpr (STAGE) {
      if (c + gridDim.x < chunks) stage(c + gridDim.x, par ^ 1);
      if (tid < D) {
        const float *m1 = &sb[par][tid * D];
        const float *r2 = &sb[par][D * D];
        float acc = 0.f;
#pragma unroll
        for (int b = 0; b < D; ++b) acc = fmaf(m1[b], r2[b], acc);
        sr[tid] = acc;
      }
    } else {
      if (tid < D) {
        const float *m1 = tab + d.m1 + ((c & mask1) * D + tid) * D;
        const float *r2 = tab + d.r2 + (c >> d.h1) * D;
        float acc = 0.f;
#pragma unroll
        for (int b = 0; b < D; ++b) acc = fmaf(m1[b], r2[b], acc);
        sr[tid] = acc;
      }
    }
    __syncthreads();
    constexpr int NM = (64 * D + WR_NT - 1) / WR_NT;  // outputs per thread
    // (unrolled only at D = 16, where independent outputs pay; at D <= 8 it would
    // cost the registers of a fourth CTA per SM)
#pragma unroll(D >= 16 ? NM : 1)
    for (int k = 0; k < NM; ++k) {
      const int i = tid + k * WR_NT;  // i = ym D + a
      if (i < 64 * D) {
        const float *mcol = sM + (i / D) * D * D + (i % D);
        float acc = 0.f;
#pragma unroll
        for (int b = 0; b < D; ++b) acc = fmaf(mcol[b * D], sr[b], acc);
        *reinterpret_cast<float2 *>(&sm[2 * i]) = make_float2(acc, acc);
      }
    }
    __syncthreads();
    float *oc = out + (c << MPS_CHUNK_BITS) + 4 * lane;
#pragma unroll 2
    for (int ym = w; ym < 64; ym += WR_NT / 32) {
      // one 16-byte broadcast load gives (m_a, m_a) and (m_{a+1}, m_{a+1});
      // even and odd a accumulate separately (shorter dependency chains)
      const ulonglong2 *mv = reinterpret_cast<const ulonglong2 *>(sm + ym * 2 * D);
      unsigned long long p01 = 0ull, p23 = 0ull, q01 = 0ull, q23 = 0ull;
#pragma unroll
      for (int a = 0; a < D; a += 2) {
        const ulonglong2 m = mv[a / 2];
        p01 = fma2(L01[a], m.x, p01);
        p23 = fma2(L23[a], m.x, p23);
        q01 = fma2(L01[a + 1], m.y, q01);
        q23 = fma2(L23[a + 1], m.y, q23);
      }
      const float2 v01 = upk(add2(p01, q01)), v23 = upk(add2(p23, q23));
      *reinterpret_cast<float4 *>(oc + ym * 128) = make_float4(v01.x, v01.y, v23.x, v23.y);
    }
  }
  if constexpr (STAGE) cp_async_wait<0>();
}

template <int D>
cudaError_t launch_mps_d(const PassArgs &A, int jobs, cudaStream_t s) {
  if (A.kind == K_MPS_TAB) {
    const MpsDims d = mps_dims(A.n, A.layer);
    const MpsItems its = mps_items(d);
    const dim3 grid((unsigned)((its.total + TAB_NT - 1) / TAB_NT), (unsigned)jobs);
    const size_t smem = (size_t)mps_tab_span(A.n, A.layer) * 2 * D * D * sizeof(double);
    if (A.em.form == EF_PREFIX) {
      if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_mps_tab<D, EF_PREFIX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_mps_tab<D, EF_PREFIX><<<grid, TAB_NT, smem, s>>>(A);
    } else {
      if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_mps_tab<D, EF_DIFF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_mps_tab<D, EF_DIFF><<<grid, TAB_NT, smem, s>>>(A);
    }
    return cudaGetLastError();
  }
  const long long cap = (long long)num_sms_cached() * (D >= 16 ? 2 : 4);
  const dim3 grid((unsigned)(A.tiles < cap ? A.tiles : cap), (unsigned)jobs);
  const size_t smem = (size_t)64 * D * D * sizeof(float);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_mps_write<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_mps_write<D><<<grid, WR_NT, smem, s>>>(A);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mps(int prec, const PassArgs &A, int jobs, cudaStream_t s) {
  if (prec != 0 || A.n < MPS_MIN_QUBITS || A.n > 30 || A.layer < 1 || A.layer > MPS_MAX_LAYERS ||
      (A.em.form != EF_DIFF && A.em.form != EF_PREFIX) || A.em.sh != 0)
    return cudaErrorInvalidValue;
  if (A.kind == K_MPS && A.tiles != (1LL << (A.n - MPS_CHUNK_BITS))) return cudaErrorInvalidValue;
  switch (A.layer) {
    case 1: return launch_mps_d<2>(A, jobs, s);
    case 2: return launch_mps_d<4>(A, jobs, s);
    case 3: return launch_mps_d<8>(A, jobs, s);
    default: return launch_mps_d<16>(A, jobs, s);
  }
}

}  // namespace gvqe
