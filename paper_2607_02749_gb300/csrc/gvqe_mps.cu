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

// Site matrix entry A_q[y](a, b) of the stage (layer r, layer r's rotated qubits
// rot), or, for dr >= 0, its derivative by layer dr's angle of qubit q: that
// layer's factor becomes d cos(t/2)/dt = -sin(t/2)/2, d sin(t/2)/dt = cos(t/2)/2.
template <int FORM>
__device__ double site_entry(const float2 *cs, int pstride, int q, int y, int a, int b, int r, bool rot,
                             int dr = -1) {
  if (q == 0 && a != 0) return 0.0;  // the left end's bond is 0
  auto bit = [](int v, int k) { return (v >> (k - 1)) & 1; };
  const float2 f = cs[q];
  const int x0 = (FORM == EF_PREFIX) ? bit(b, 1) : (bit(b, 1) ^ bit(a, 1));
  double v = (dr == 0) ? (x0 ? 0.5 * (double)f.x : -0.5 * (double)f.y) : (x0 ? (double)f.y : (double)f.x);
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
    const float2 g = cs[(size_t)k * pstride + q];
    if (k == dr)
      v *= (out == in) ? -0.5 * (double)g.y : (out ? 0.5 * (double)g.x : -0.5 * (double)g.x);
    else
      v *= ry_entry(g, out, in);
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
  const long long row_blocks = (its.total + TAB_NT - 1) / TAB_NT;
  if (blockIdx.x >= row_blocks) {
    // the site matrices [q][y][a][b] and their derivatives [k][q][y][a][b], one entry per thread
    const long long e = (blockIdx.x - row_blocks) * TAB_NT + tid;
    const long long ns = (long long)n * 2 * DD;
    if (e >= ns * (r + 2)) return;
    const int k = (int)(e / ns) - 1;  // -1: the matrices themselves
    const long long w = e % ns;
    const int b = (int)(w % D), a = (int)((w / D) % D), y = (int)((w / DD) & 1), q = (int)(w / (2 * DD));
    const bool rot = (A.gate_mask >> q) & 1u;
    const double v = (FORM == EF_PREFIX) ? site_entry<EF_PREFIX>(cs, A.pstride, q, y, a, b, r, rot, k)
                                         : site_entry<EF_DIFF>(cs, A.pstride, q, y, a, b, r, rot, k);
    float *tab = reinterpret_cast<float *>(A.out) + (size_t)job * A.out_stride;
    tab[d.sites + e] = (float)v;  // d.dsites = d.sites + ns
    return;
  }
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
  constexpr int MS_LD = D * D + D;  // per-ym stride: the lanes of m = M R_c cross ym on distinct banks
  extern __shared__ __align__(16) float sM[];  // [64][b][a] (transposed), MS_LD floats per ym, dynamic
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
    sM[ym * MS_LD + b * D + a] = tab[d.mid + (ym * D + a) * D + b];
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
        const float *mcol = sM + (i / D) * MS_LD + (i % D);
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

// ------------------------------------------------- closed-form gradients --
// For the angles of layers 0..r (the closed-form ones), with lambda_r the
// adjoint state at the output of layer r (the backward passes of layers
// D..r+1 bring it there),
//
//   dE/dtheta_{k,q} = 2 <lambda_r | d psi_r / d theta_{k,q}>,
//
// and d psi_r / d theta_{k,q} is the same matrix product with site q's matrix
// replaced by its derivative dA_q^k.  Split psi_r(y) = L(y_0..6) M(y_7..12) R_c
// (R_c = the column vector of the chunk's high qubits), and contract lambda
// once, chunk by chunk (k_mps_grad):
//   mu(y_0..6)  = sum over chunks and y_7..12 of lambda(y) M(y_7..12) R_c  (row-side qubits 0..6)
//   P(y_7..12)  = sum over chunks of [sum_{y_0..6} lambda(y) L(y_0..6)] (x) R_c  (qubits 7..12)
//   l_c         = sum_{y_0..12} lambda(y) L(y_0..6) M(y_7..12)  (one row vector per chunk)
// Then qubits 0..12 take their gradients from mu and P (k_mps_genv), and the
// high qubits from l_c, per chunk: l_c A_13 .. dA_q .. A_{n-1} 1 (k_mps_ghigh).
// Sums run in FP32 inside a chunk (a thread's 32 rows or columns, the four
// column quarters) and over 8 chunks, then in FP64 across chunks and CTAs, in
// a fixed order.

constexpr int GR_NT = 256;
constexpr int LAM_LD = 132;  // floats per staged lambda row (128 + 4: 16-byte aligned, see k_mps_grad)

// One pass over lambda_r, chunk by chunk, each chunk's 64 x 128 lambda block
// (rows: qubits 7..12, columns: qubits 0..6) staged in shared memory by
// cp.async while the previous chunk is contracted.  Per chunk, with m = M R_c
// as in the writer:
//   Lambda1 = lambda_c L     (64 x D; thread (k-quarter, row) keeps one row's D sums
//                             over 32 columns, the quarters are added in shared memory)
//   mu     += lambda_c^T m   (128 x D; thread (half, column) keeps one column's D sums
//                             over 32 rows, in registers across chunks)
//   P      += Lambda1 (x) R_c,  l_c = sum_rows Lambda1(row) M(row)
// Both products read the block conflict-free: rows are 132 floats apart and the
// k order of the Lambda1 product is rotated per lane (lane 8i + j starts at
// column offset i, so bank 4j + i + k differs across the warp).  Every 8 chunks
// the FP32 accumulators are added into this CTA's FP64 partials.
template <int D>
__global__ void __launch_bounds__(GR_NT, 2) k_mps_grad(const PassArgs A) {
  // dynamic: two staged lambda blocks, the transposed mid matrices [64][b][a],
  // the row vectors of qubits 0..6 [128][D], then quarter partials [4][64][D]
  // (D <= 8) or the P accumulators [64][D][D] (D = 16, too many for registers)
  extern __shared__ __align__(16) float dyn[];
  constexpr bool BIG = D >= 16;
  float *slam = dyn;                        // [2][64][LAM_LD]
  constexpr int MS_LD = D * D + D;          // per-ym stride of the transposed mid matrices
  float *sM = slam + 2 * 64 * LAM_LD;       // [64][MS_LD]: [b][a]
  float *sLo = sM + 64 * MS_LD;             // [128][D]
  float *sQ = sLo + 128 * D;                // [4][64][D] (D <= 8)
  float *sP = sLo + 128 * D;                // [64][D][D] (D = 16)
  __shared__ __align__(16) float sm[64 * D];  // m per row (8-byte pairs read as f32x2)
  __shared__ __align__(16) float sb[2][D * D + D];
  __shared__ float sr[D];
  __shared__ float sL1[64 * D];
  __shared__ float sLc[GR_NT / 32][D];
  constexpr bool STAGE = D >= 4;  // the chunk's matrix and vector by cp.async (16-byte pieces)
  constexpr int NCH = (D * D + D) / 4;
  constexpr int NP = (64 * D * D) / GR_NT;  // P entries per thread
  constexpr int NPR = BIG ? 1 : NP;         // ... held in registers (D <= 8)
  constexpr int FLUSH = 8;
  const int r = (D == 2) ? 1 : (D == 4 ? 2 : (D == 8 ? 3 : 4));
  const MpsDims d = mps_dims(A.n, r);
  const MpsGradRegions gr = mps_grad_regions(A.n, r);
  const int job = blockIdx.y, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const float *tab = reinterpret_cast<const float *>(A.in) + (size_t)job * A.in_stride;
  const float *lam = reinterpret_cast<const float *>(A.lam_in) + (size_t)job * A.lam_stride;
  double *part = A.part + (size_t)job * A.part_stride + (size_t)blockIdx.x * gr.v1;
  float *lall = reinterpret_cast<float *>(A.out) + (size_t)job * A.out_stride;
  const long long chunks = A.tiles;
  const long long mask1 = (1LL << d.h1) - 1;
  // mu (partial layout [a][128]): D <= 8, thread (half h, column u) sums rows
  // [32 h, 32 h + 32) of column u for every a; D = 16, thread (a-half h, column u)
  // sums every row for a in [8 h, 8 h + 8)
  const int mh = tid >> 7, mu_col = tid & 127;
  // Lambda1: D <= 8, thread (quarter qt, row ym) sums columns [32 qt, 32 qt + 32)
  // of row ym; D = 16, thread (row, a-quarter) sums every column for 4 of the a
  const int qt = tid >> 6, l1_row = tid & 63, rot = (l1_row >> 3) & 3;
  const int b_row = tid >> 2, b_aq = tid & 3;
  if constexpr (BIG) {
#pragma unroll
    for (int j = 0; j < D / 2; ++j) part[(size_t)(mh * (D / 2) + j) * 128 + mu_col] = 0.0;
  } else if (mh == 0) {
#pragma unroll
    for (int a = 0; a < D; ++a) part[(size_t)a * 128 + mu_col] = 0.0;
  }
#pragma unroll
  for (int k = 0; k < NP; ++k) part[128 * D + tid + GR_NT * k] = 0.0;
  if constexpr (BIG) {
#pragma unroll
    for (int k = 0; k < NP; ++k) sP[tid + GR_NT * k] = 0.f;
  }
  // chunk c's staged data into buffer buf: its matrix of [13, 13 + h1) and vector
  // of [13 + h1, n), and its 64 x 128 lambda block
  auto stage = [&](long long c, int buf) {
    if (STAGE && tid < NCH) {
      const float *src = (tid < D * D / 4) ? tab + d.m1 + (c & mask1) * D * D + 4 * tid
                                           : tab + d.r2 + (c >> d.h1) * D + 4 * (tid - D * D / 4);
      cp_async16(&sb[buf][4 * tid], src);
    }
    const float *lc = lam + (c << MPS_CHUNK_BITS);
    float *dst = slam + buf * 64 * LAM_LD;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int i = tid + GR_NT * j, row = i >> 5, col = (i & 31) * 4;
      cp_async16(dst + row * LAM_LD + col, lc + row * 128 + col);
    }
    cp_async_commit();
  };
  stage(blockIdx.x, 0);
  for (int i = tid; i < 64 * D * D; i += GR_NT) {
    const int ym = i / (D * D), b = (i / D) % D, a = i % D;
    sM[ym * MS_LD + b * D + a] = tab[d.mid + (ym * D + a) * D + b];
  }
  for (int i = tid; i < 128 * D; i += GR_NT) sLo[i] = tab[d.lo + (i % D) * 128 + i / D];  // [yl][a]
  constexpr int NMU2 = BIG ? D / 4 : D / 2;
  unsigned long long mu2[NMU2];  // packed pairs of this thread's mu values
  float Pacc[NPR];
#pragma unroll
  for (int a = 0; a < NMU2; ++a) mu2[a] = 0ull;
#pragma unroll
  for (int k = 0; k < NPR; ++k) Pacc[k] = 0.f;
  auto flush_big = [&]() {
#pragma unroll
    for (int j = 0; j < NMU2; ++j) {
      const float2 m = upk(mu2[j]);
      part[(size_t)(mh * (D / 2) + 2 * j) * 128 + mu_col] += (double)m.x;
      part[(size_t)(mh * (D / 2) + 2 * j + 1) * 128 + mu_col] += (double)m.y;
      mu2[j] = 0ull;
    }
#pragma unroll 8
    for (int k = 0; k < NP; ++k) {
      part[128 * D + tid + GR_NT * k] += (double)sP[tid + GR_NT * k];
      sP[tid + GR_NT * k] = 0.f;
    }
  };
  auto flush = [&]() {
    // the two row halves of each column meet in sQ (free at this point)
    if (mh == 1) {
#pragma unroll
      for (int a = 0; a < D / 2; ++a) {
        const float2 m = upk(mu2[a]);
        sQ[(2 * a) * 128 + mu_col] = m.x;
        sQ[(2 * a + 1) * 128 + mu_col] = m.y;
      }
    }
    __syncthreads();
    if (mh == 0) {
#pragma unroll
      for (int a = 0; a < D / 2; ++a) {
        const float2 m = upk(mu2[a]);
        part[(size_t)(2 * a) * 128 + mu_col] += (double)(m.x + sQ[(2 * a) * 128 + mu_col]);
        part[(size_t)(2 * a + 1) * 128 + mu_col] += (double)(m.y + sQ[(2 * a + 1) * 128 + mu_col]);
      }
    }
#pragma unroll
    for (int a = 0; a < D / 2; ++a) mu2[a] = 0ull;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      part[128 * D + tid + GR_NT * k] += (double)Pacc[k];
      Pacc[k] = 0.f;
    }
    __syncthreads();  // sQ free again
  };
  int par = 0, since = 0;
  for (long long c = blockIdx.x; c < chunks; c += gridDim.x, par ^= 1) {
    cp_async_wait<0>();
    __syncthreads();  // chunk c staged; the previous chunk's shared vectors are read
    if (c + gridDim.x < chunks) stage(c + gridDim.x, par ^ 1);
    if (tid < D) {
      float acc = 0.f;
      if constexpr (STAGE) {
#pragma unroll
        for (int b = 0; b < D; ++b) acc = fmaf(sb[par][tid * D + b], sb[par][D * D + b], acc);
      } else {
        const float *m1 = tab + d.m1 + ((c & mask1) * D + tid) * D;
        const float *r2 = tab + d.r2 + (c >> d.h1) * D;
#pragma unroll
        for (int b = 0; b < D; ++b) acc = fmaf(m1[b], r2[b], acc);
      }
      sr[tid] = acc;
    }
    __syncthreads();
    for (int i = tid; i < 64 * D; i += GR_NT) {
      const float *mcol = sM + (i / D) * MS_LD + (i % D);
      float acc = 0.f;
#pragma unroll
      for (int b = 0; b < D; ++b) acc = fmaf(mcol[b * D], sr[b], acc);
      sm[i] = acc;
    }
    __syncthreads();
    const float *blk = slam + par * 64 * LAM_LD;
    if constexpr (BIG) {
      // mu += lambda^T m: column mu_col, every row, a in [8 mh, 8 mh + 8)
      const float *col = blk + mu_col;
#pragma unroll 4
      for (int ym = 0; ym < 64; ++ym) {
        const float l = col[ym * LAM_LD];
        const unsigned long long l2 = pk(l, l);
        const unsigned long long *mv = reinterpret_cast<const unsigned long long *>(sm + ym * D + mh * (D / 2));
#pragma unroll
        for (int j = 0; j < NMU2; ++j) mu2[j] = fma2(l2, mv[j], mu2[j]);
      }
      // Lambda1 row b_row, a in [4 b_aq, 4 b_aq + 4), every column (rows 132 floats
      // apart: the warp's 8 rows fall in distinct banks)
      unsigned long long acc[2] = {0ull, 0ull};
      const float *row = blk + b_row * LAM_LD;
#pragma unroll 4
      for (int k = 0; k < 128; ++k) {
        const float l = row[k];
        const unsigned long long l2 = pk(l, l);
        const unsigned long long *lv = reinterpret_cast<const unsigned long long *>(sLo + k * D + 4 * b_aq);
        acc[0] = fma2(l2, lv[0], acc[0]);
        acc[1] = fma2(l2, lv[1], acc[1]);
      }
      *reinterpret_cast<float2 *>(&sL1[b_row * D + 4 * b_aq]) = upk(acc[0]);
      *reinterpret_cast<float2 *>(&sL1[b_row * D + 4 * b_aq + 2]) = upk(acc[1]);
      __syncthreads();
    } else {
    {
      // mu += lambda^T m over this thread's 32 rows (packed pairs of bond indices)
      const float *col = blk + mu_col;
#pragma unroll 4
      for (int k = 0; k < 32; ++k) {
        const int ym = 32 * mh + k;
        const float l = col[ym * LAM_LD];
        const unsigned long long l2 = pk(l, l);
        const unsigned long long *mv = reinterpret_cast<const unsigned long long *>(sm + ym * D);
#pragma unroll
        for (int a = 0; a < D / 2; ++a) mu2[a] = fma2(l2, mv[a], mu2[a]);
      }
    }
    {
      // Lambda1 quarter sums: row l1_row, columns 32 qt + (k + rot) mod 32
      unsigned long long acc[D / 2];
#pragma unroll
      for (int a = 0; a < D / 2; ++a) acc[a] = 0ull;
      const float *row = blk + l1_row * LAM_LD + 32 * qt;
      const float *lo = sLo + 32 * qt * D;
#pragma unroll 4
      for (int k = 0; k < 32; ++k) {
        const int yl = (k + rot) & 31;
        const float l = row[yl];
        const unsigned long long l2 = pk(l, l);
        const unsigned long long *lv = reinterpret_cast<const unsigned long long *>(lo + yl * D);
#pragma unroll
        for (int a = 0; a < D / 2; ++a) acc[a] = fma2(l2, lv[a], acc[a]);
      }
#pragma unroll
      for (int a = 0; a < D / 2; ++a)
        *reinterpret_cast<float2 *>(&sQ[(qt * 64 + l1_row) * D + 2 * a]) = upk(acc[a]);
    }
    __syncthreads();
    for (int i = tid; i < 64 * D; i += GR_NT) sL1[i] = sQ[i] + sQ[64 * D + i] + sQ[128 * D + i] + sQ[192 * D + i];
    __syncthreads();
    }
    if constexpr (BIG) {
#pragma unroll 8
      for (int k = 0; k < NP; ++k) {
        const int e = tid + GR_NT * k;  // (ym D + a) D + b
        sP[e] = fmaf(sL1[e / D], sr[e % D], sP[e]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const int e = tid + GR_NT * k;  // (ym D + a) D + b
        Pacc[k] = fmaf(sL1[e / D], sr[e % D], Pacc[k]);
      }
    }
    {
      // l_c(b) = sum over (ym, a) of sL1[ym][a] M(ym)(a, b): thread (g, b) takes every
      // (GR_NT / D)-th (ym, a), then the warp and the CTA sum over g
      const int b = tid % D, g = tid / D;
      float x = 0.f;
      for (int i = g; i < 64 * D; i += GR_NT / D) x = fmaf(sL1[i], sM[(i / D) * MS_LD + b * D + (i % D)], x);
#pragma unroll
      for (int off = D; off < 32; off <<= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
      if (lane < D) sLc[w][lane] = x;
    }
    __syncthreads();
    if (tid < D) {
      float t = 0.f;
#pragma unroll
      for (int ww = 0; ww < GR_NT / 32; ++ww) t += sLc[ww][tid];
      lall[c * D + tid] = t;
    }
    if (++since == FLUSH) {
      if constexpr (BIG)
        flush_big();
      else
        flush();
      since = 0;
    }
  }
  if (since > 0) {
    if constexpr (BIG)
      flush_big();
    else
      flush();
  }
  cp_async_wait<0>();
}

// Bond dimension 16: the same pass, 16 warps per CTA and one CTA per SM.
// Warps 0..7 form Lambda1: thread (row, column quarter) over 32 columns for
// all 16 a, four columns per 16-byte load (rows 132 floats apart keep a
// quarter-warp's rows in distinct banks), the quarters added in shared memory.  Warps 8..15 form
// mu: thread (column pair, a-half, row half) over 32 rows, two columns per
// 8-byte load.  P lives in registers (thread: two (row, a) pairs x 16 b), and
// l_c is summed with it from the same Lambda1 values and rows of the mid
// matrices.  The shared loads are 16-byte vectors wherever the lanes allow, so
// the shared-memory pipe, not the FMA pipe, sets the pace.  FP32 accumulators
// are added into the FP64 partials every 16 chunks.
constexpr int G16_NT = 512;
constexpr int G16_RS = 20;  // floats per 16-float row of the mid matrices and the quarters (16 + 4)
__global__ void __launch_bounds__(G16_NT, 1) k_mps_grad16(const PassArgs A) {
  constexpr int D = 16, DD = 256;
  // 16-float rows read or written by consecutive lanes sit G16_RS floats apart:
  // eight lanes' 16-byte accesses then fall in eight distinct bank groups
  extern __shared__ __align__(16) float dyn[];
  float *slam = dyn;                    // [2][64][LAM_LD]
  float *sMn = slam + 2 * 64 * LAM_LD;  // [64 D rows (ym, a)][G16_RS]: M(ym)(a, b)
  float *sLo = sMn + 64 * D * G16_RS;   // [128][D]
  float *sQ = sLo + 128 * D;            // [4 x 64 rows][G16_RS]: Lambda1 quarters; mu row halves at a flush
  __shared__ __align__(16) float sm[64 * D];
  __shared__ __align__(16) float sb[2][DD + D];
  __shared__ __align__(16) float sr[D];
  __shared__ __align__(16) float sL1[64 * D];
  __shared__ float sLc[G16_NT / 32][D];
  constexpr int NCH = (DD + D) / 4;
  constexpr int FLUSH = 16;
  const MpsDims d = mps_dims(A.n, 4);
  const MpsGradRegions gr = mps_grad_regions(A.n, 4);
  const int job = blockIdx.y, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const float *tab = reinterpret_cast<const float *>(A.in) + (size_t)job * A.in_stride;
  const float *lam = reinterpret_cast<const float *>(A.lam_in) + (size_t)job * A.lam_stride;
  double *part = A.part + (size_t)job * A.part_stride + (size_t)blockIdx.x * gr.v1;
  float *lall = reinterpret_cast<float *>(A.out) + (size_t)job * A.out_stride;
  const long long chunks = A.tiles;
  const long long mask1 = (1LL << d.h1) - 1;
  const bool l1w = tid < 256;
  const int t2 = tid & 255;
  // Lambda1 warps: thread (row l_row, column quarter l_q) sums columns
  // [32 l_q, 32 l_q + 32) for all 16 a; a warp's lanes take 32 consecutive rows
  const int l_row = t2 & 63, l_q = t2 >> 6;
  // mu warps: column pair (t2 & 63), a-half ((t2 >> 6) & 1), row half (t2 >> 7)
  const int m_cp = t2 & 63, m_ah = (t2 >> 6) & 1, m_rh = t2 >> 7;
  if (!l1w && m_rh == 0) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      part[(size_t)(8 * m_ah + j) * 128 + 2 * m_cp] = 0.0;
      part[(size_t)(8 * m_ah + j) * 128 + 2 * m_cp + 1] = 0.0;
    }
  }
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int b = 0; b < D; ++b) part[128 * D + (size_t)(tid + G16_NT * p) * D + b] = 0.0;
  auto stage = [&](long long c, int buf) {
    if (tid < NCH) {
      const float *src = (tid < DD / 4) ? tab + d.m1 + (c & mask1) * DD + 4 * tid
                                        : tab + d.r2 + (c >> d.h1) * D + 4 * (tid - DD / 4);
      cp_async16(&sb[buf][4 * tid], src);
    }
    const float *lc = lam + (c << MPS_CHUNK_BITS);
    float *dst = slam + buf * 64 * LAM_LD;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int i = tid + G16_NT * j, row = i >> 5, col = (i & 31) * 4;
      cp_async16(dst + row * LAM_LD + col, lc + row * 128 + col);
    }
    cp_async_commit();
  };
  stage(blockIdx.x, 0);
  for (int i = tid; i < 64 * DD; i += G16_NT) sMn[(i / D) * G16_RS + i % D] = tab[d.mid + i];
  for (int i = tid; i < 128 * D; i += G16_NT) sLo[i] = tab[d.lo + (i % D) * 128 + i / D];  // [yl][a]
  // mu: 2 columns x 8 a (packed pairs over a); P: 2 pairs x 16 b (packed pairs over b)
  unsigned long long mu2[2][4], P2[2][8];
#pragma unroll
  for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
    for (int j = 0; j < 4; ++j) mu2[c2][j] = 0ull;
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int j = 0; j < 8; ++j) P2[p][j] = 0ull;
  auto flush = [&]() {
    // mu: the row-half-1 threads park their sums in sQ, the row-half-0 threads add both
    // parked as [a (8)][column of the pair][a-half][column pair]: consecutive lanes, consecutive words
    auto park = [&](int jj, int c2) { return ((jj * 2 + c2) * 2 + m_ah) * 64 + m_cp; };
    if (!l1w && m_rh == 1) {
#pragma unroll
      for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float2 m = upk(mu2[c2][j]);
          sQ[park(2 * j, c2)] = m.x;
          sQ[park(2 * j + 1, c2)] = m.y;
        }
    }
    __syncthreads();
    if (!l1w && m_rh == 0) {
#pragma unroll
      for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float2 m = upk(mu2[c2][j]);
          part[(size_t)(8 * m_ah + 2 * j) * 128 + 2 * m_cp + c2] += (double)(m.x + sQ[park(2 * j, c2)]);
          part[(size_t)(8 * m_ah + 2 * j + 1) * 128 + 2 * m_cp + c2] += (double)(m.y + sQ[park(2 * j + 1, c2)]);
        }
    }
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
      for (int j = 0; j < 4; ++j) mu2[c2][j] = 0ull;
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float2 v = upk(P2[p][j]);
        double *dst = part + 128 * D + (size_t)(tid + G16_NT * p) * D + 2 * j;
        dst[0] += (double)v.x;
        dst[1] += (double)v.y;
        P2[p][j] = 0ull;
      }
    __syncthreads();  // sQ free for the next chunk's quarters
  };
  int par = 0, since = 0;
  for (long long c = blockIdx.x; c < chunks; c += gridDim.x, par ^= 1) {
    cp_async_wait<0>();
    __syncthreads();
    if (c + gridDim.x < chunks) stage(c + gridDim.x, par ^ 1);
    if (tid < D) {
      float acc = 0.f;
#pragma unroll
      for (int b = 0; b < D; ++b) acc = fmaf(sb[par][tid * D + b], sb[par][DD + b], acc);
      sr[tid] = acc;
    }
    __syncthreads();
    {
      // m(ym)(a) = M(ym)(a, :) R_c: thread (ym, a) for two rows, 16-byte row loads
      const float4 *r4 = reinterpret_cast<const float4 *>(sr);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int i = tid + G16_NT * k;  // ym D + a
        const float4 *mrow = reinterpret_cast<const float4 *>(sMn + (size_t)i * G16_RS);
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float4 m = mrow[j], rr = r4[j];
          acc = fmaf(m.x, rr.x, fmaf(m.y, rr.y, fmaf(m.z, rr.z, fmaf(m.w, rr.w, acc))));
        }
        sm[i] = acc;
      }
    }
    __syncthreads();
    const float *blk = slam + par * 64 * LAM_LD;
    if (l1w) {
      // Lambda1 quarter: row l_row, columns [32 l_q, 32 l_q + 32), all 16 a
      unsigned long long acc[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] = 0ull;
      const float4 *row4 = reinterpret_cast<const float4 *>(blk + l_row * LAM_LD + 32 * l_q);
      const ulonglong2 *lo2 = reinterpret_cast<const ulonglong2 *>(sLo + 32 * l_q * D);
#pragma unroll 2
      for (int k4 = 0; k4 < 8; ++k4) {
        const float4 l4 = row4[k4];
        const float lv[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const unsigned long long l2 = pk(lv[e], lv[e]);
          const ulonglong2 *lr = lo2 + (4 * k4 + e) * (D / 4);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const ulonglong2 v = lr[j];
            acc[2 * j] = fma2(l2, v.x, acc[2 * j]);
            acc[2 * j + 1] = fma2(l2, v.y, acc[2 * j + 1]);
          }
        }
      }
      float4 *q4 = reinterpret_cast<float4 *>(sQ + (l_q * 64 + l_row) * G16_RS);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 x = upk(acc[2 * j]), y = upk(acc[2 * j + 1]);
        q4[j] = make_float4(x.x, x.y, y.x, y.y);
      }
    } else {
      // mu: columns 2 m_cp, 2 m_cp + 1; rows [32 m_rh, 32 m_rh + 32); a in [8 m_ah, 8 m_ah + 8)
      const float *colp = blk + 2 * m_cp;
#pragma unroll 4
      for (int k = 0; k < 32; ++k) {
        const int ym = 32 * m_rh + k;
        const float2 l = *reinterpret_cast<const float2 *>(colp + ym * LAM_LD);
        const unsigned long long lx = pk(l.x, l.x), ly = pk(l.y, l.y);
        const ulonglong2 *mv = reinterpret_cast<const ulonglong2 *>(sm + ym * D + 8 * m_ah);
        const ulonglong2 m0 = mv[0], m1 = mv[1];
        mu2[0][0] = fma2(lx, m0.x, mu2[0][0]);
        mu2[0][1] = fma2(lx, m0.y, mu2[0][1]);
        mu2[0][2] = fma2(lx, m1.x, mu2[0][2]);
        mu2[0][3] = fma2(lx, m1.y, mu2[0][3]);
        mu2[1][0] = fma2(ly, m0.x, mu2[1][0]);
        mu2[1][1] = fma2(ly, m0.y, mu2[1][1]);
        mu2[1][2] = fma2(ly, m1.x, mu2[1][2]);
        mu2[1][3] = fma2(ly, m1.y, mu2[1][3]);
      }
    }
    __syncthreads();
    // Lambda1 = the sum of the four column quarters
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int i = tid + G16_NT * k, o = (i / D) * G16_RS + i % D;  // row ym = i / D, a = i % D
      sL1[i] = sQ[o] + sQ[64 * G16_RS + o] + sQ[128 * G16_RS + o] + sQ[192 * G16_RS + o];
    }
    __syncthreads();
    {
      // P(pair, :) += Lambda1(pair) R_c and l_c(:) += Lambda1(pair) M(pair)(:), for two pairs
      const ulonglong2 *rv = reinterpret_cast<const ulonglong2 *>(sr);
      unsigned long long lc2[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) lc2[j] = 0ull;
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int pair = tid + G16_NT * p;  // ym D + a
        const float L = sL1[pair];
        const unsigned long long L2 = pk(L, L);
        const ulonglong2 *mr = reinterpret_cast<const ulonglong2 *>(sMn + (size_t)pair * G16_RS);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const ulonglong2 rr = rv[j], mm = mr[j];
          P2[p][2 * j] = fma2(L2, rr.x, P2[p][2 * j]);
          P2[p][2 * j + 1] = fma2(L2, rr.y, P2[p][2 * j + 1]);
          lc2[2 * j] = fma2(L2, mm.x, lc2[2 * j]);
          lc2[2 * j + 1] = fma2(L2, mm.y, lc2[2 * j + 1]);
        }
      }
      // sum the 16 values of l_c over the warp (transposed halving: 8 + 4 + 2 + 1 exchanges)
      float v[16];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float2 t = upk(lc2[j]);
        v[2 * j] = t.x;
        v[2 * j + 1] = t.y;
      }
      int cnt = 16;
#pragma unroll
      for (int sh = 16; sh >= 2; sh >>= 1) {
        const int half = cnt / 2;
        const bool hi = (lane & sh) != 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (j < half) {
            const float keep = hi ? v[half + j] : v[j];
            const float send = hi ? v[j] : v[half + j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, sh);
          }
        }
        cnt = half;
      }
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
      // lane bits 4..1 name the value: b = 8 b4 + 4 b3 + 2 b2 + b1
      if ((lane & 1) == 0) {
        const int b = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
        sLc[w][b] = v[0];
      }
    }
    __syncthreads();
    if (tid < D) {
      float t = 0.f;
#pragma unroll
      for (int ww = 0; ww < G16_NT / 32; ++ww) t += sLc[ww][tid];
      lall[c * D + tid] = t;
    }
    if (++since == FLUSH) {
      flush();
      since = 0;
    }
  }
  if (since > 0) flush();
  cp_async_wait<0>();
}

// ------------------------------------------------ bond 16 on the tensor cores --
// The two contractions of the bond-16 pass that grow with the chunk,
// Lambda1 = lambda_c L (64 x 128 by 128 x 16) and mu += lambda_c^T m
// (128 x 64 by 64 x 16), run as tcgen05.mma kind::tf32 with FP32 accumulators
// in tensor memory.  TF32 keeps 10 mantissa bits, so every operand x is split
// into x_hi (x with its low 13 mantissa bits cleared) and x_lo = x - x_hi
// (four-term split products, relative error about 2^-21 per product, the level
// of the FP32 SIMT pass): Lambda1 takes A = [lambda_hi; lambda_lo] (128 rows)
// against B = [L_hi | L_lo] (N = 32) in one 128 x 32 accumulator, whose four
// 64 x 16 blocks add up to Lambda1; mu takes A = lambda_hi^T, then lambda_lo^T,
// against B = [m_hi | m_lo] into a 128 x 32 accumulator, whose two column halves
// add up to mu: 16 + 16 MMAs (M = 128, N = 32, K = 8) per chunk.  Both contractions read lambda
// with K-major operands (the MN-major operand form gave zeros for TF32 on
// sm_103a), so each chunk's split lambda is written twice: rows ym
// with runs of yl for Lambda1, rows yl with runs of ym for mu.  Operand
// layout: no swizzle, core matrices of 8 rows x 16 bytes; LBO steps along K,
// SBO along the rows.  The K strides are padded (144 bytes between the
// Lambda1 core matrices along yl, 2064 bytes between 8-row groups of the mu
// copy) so that the split writes, one 4 x 4 block per thread, are free of
// bank conflicts.
//
// The rest stays on the FP32 pipe: R_c, m = M R_c and, for the previous chunk
// while the tensor cores work on this one, P += Lambda1 (x) R_c and
// l_c = sum Lambda1 M (each thread keeps its two rows of the mid matrices in
// registers for the whole pass).  Each chunk's mu starts afresh in tensor memory
// and is added, in FP32 with round-to-nearest, into a shared-memory sum (the
// tensor cores' own accumulation over many chunks drifted: 9e-6 relative after
// 32 chunks against 2e-7 on the FP32 pipe); every FLUSH chunks that sum and P
// are added into the FP64 partials.
//
// Pipeline.  lambda is copied (cp.async) straight into the Lambda1 operand
// layout: those FP32 values are lambda_hi as the tensor cores read them (the
// top 19 bits), so only lambda_lo and the mu copy are written by the threads.
// The copy buffer is double: [hi 0 | lo | hi 1], and chunk parity 0 stacks
// [hi 0; lo], parity 1 [lo; hi 1] (either way Lambda1 is the sum of the two
// 64-row halves).  Lambda1's accumulator is double too.  One thread issues
// each chunk's MMAs in two commits, Lambda1 (mbarrier barL) and mu (barM), so
// that lambda_lo of chunk c + 1 is written while mu(c) runs and the mu copy of
// c + 1 while Lambda1(c + 1) runs; the previous chunk's Lambda1 rows are read
// out and its P and l_c formed meanwhile.  Three CTA barriers per chunk.
//
// Every thread waits on the mbarriers with a bounded spin.  A wait that runs
// out (not expected: the MMAs always complete) writes NaN into the CTA's
// partials, so the job's gradients come out NaN, and frees tensor memory only
// once both mbarriers report their last commit complete.
constexpr int TC_NT = 512;
constexpr int TC_FLUSH = 32;
// float offsets of the shared-memory regions
constexpr int TC_HALF = 8 * 1152;         // 64 rows of the Lambda1 operand: 8 groups x 4608 bytes
constexpr int TC_A1 = 0;                  // lambda for Lambda1: [hi 0 | lo | hi 1]
constexpr int TC_AT = TC_A1 + 3 * TC_HALF;  // lambda^T for mu: hi, lo, 16 groups x 2064 bytes each
constexpr int TC_LB = TC_AT + 2 * 8256;   // [L_hi | L_lo] (B of Lambda1: 32 rows x 128 yl), 16 KB
constexpr int TC_MB = TC_LB + 4096;       // [m_hi | m_lo] (B of mu: 32 rows x 64 ym), 8 KB
constexpr int TC_Q = TC_MB + 2048;        // Lambda1 rows from tensor memory: 128 x 20
constexpr int TC_SB = TC_Q + 128 * 20;    // staged M_h1 and r_h2: [2][272]
constexpr int TC_SR = TC_SB + 2 * 272;    // R_c: [2][16]
constexpr int TC_LC = TC_SR + 32;         // l_c per warp: [16][16]
constexpr int TC_MU = TC_LC + 256;        // mu summed over chunks in FP32: [128 yl][20]
constexpr int TC_BAR = TC_MU + 128 * 20;  // mbarriers barL, barM (8 bytes each), the tensor-memory address
constexpr size_t TC_SMEM = (size_t)(TC_BAR + 8) * sizeof(float);
static_assert(TC_SMEM <= 232448, "the bond-16 tensor-core pass needs at most 227 KB of shared memory");

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
// shared-memory matrix descriptor: start address, LBO and SBO in 16-byte units,
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// instruction descriptor: FP32 accumulator, TF32 A and B, both K-major, M = 128, N = 32
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
// the two parts of x: hi keeps the sign, exponent and top 10 mantissa bits (a TF32
// value), lo = x - hi exactly; the tensor cores read lo's top 19 bits, so lo loses
// under 2^-11 of itself, about 2^-21 of x
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc));
}
__device__ __forceinline__ void tc_ld16(uint32_t ta, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(ta)
      : "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < (1 << 22) && !done; ++it)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
  return done != 0;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__global__ void __launch_bounds__(TC_NT, 1) k_mps_grad16tc(const PassArgs A) {
  constexpr int D = 16, DD = 256;
  extern __shared__ __align__(16) float dyn[];
  float *sAT = dyn + TC_AT, *sQ = dyn + TC_Q, *sb = dyn + TC_SB, *sr = dyn + TC_SR, *sLc = dyn + TC_LC;
  float *sMu = dyn + TC_MU;
  const uint32_t barL = smem_u32(dyn + TC_BAR), barM = barL + 8;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(dyn + TC_BAR + 4);
  const MpsDims d = mps_dims(A.n, 4);
  const MpsGradRegions gr = mps_grad_regions(A.n, 4);
  const int job = blockIdx.y, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const float *tab = reinterpret_cast<const float *>(A.in) + (size_t)job * A.in_stride;
  const float *lam = reinterpret_cast<const float *>(A.lam_in) + (size_t)job * A.lam_stride;
  double *part = A.part + (size_t)job * A.part_stride + (size_t)blockIdx.x * gr.v1;
  float *lall = reinterpret_cast<float *>(A.out) + (size_t)job * A.out_stride;
  const long long chunks = A.tiles;
  const long long mask1 = (1LL << d.h1) - 1;
  // rows of the mid matrices (pairs (ym, a), index 16 ym + a) owned by this thread
  const int pr0 = 128 * (w >> 2) + 32 * (w & 3) + lane;
  // the serial jobs sit in different warps, so that no warp reaches the CTA barriers late
  // with all of them: MMA issue (warp 0, lane 0), Lambda1 readout and mu flush (warps 4..7,
  // one per tensor-memory lane quarter), R_c (warp 8), the l_c sums (warp 9)
  const bool issuer = tid == 0, rw = (w >> 2) == 1;
  const int rc_t = tid - 8 * 32, ls_t = tid - 9 * 32;
#pragma unroll
  for (int k = 0; k < 4; ++k) part[tid + TC_NT * k] = 0.0;  // mu: [a][yl]
  for (int i = tid; i < 128 * 20; i += TC_NT) sMu[i] = 0.f;
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int b = 0; b < D; ++b) part[128 * D + (size_t)(pr0 + 512 * p) * D + b] = 0.0;
  // [L_hi | L_lo]: rows a (L_lo two 8-row groups on), runs of 4 yl; L(yl, a) = tab[lo + 128 a + yl]
  for (int i = tid; i < 128 * D; i += TC_NT) {
    const int a = i >> 7, yl = i & 127;
    const float x = tab[d.lo + i], h = tf32_hi(x);
    const int o = (a >> 3) * 1024 + (yl >> 2) * 32 + (a & 7) * 4 + (yl & 3);
    dyn[TC_LB + o] = h;
    dyn[TC_LB + 2048 + o] = x - h;
  }
  unsigned long long Mr[2][8];  // M(ym)(a, b) for this thread's two pairs, packed over b
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const float4 *src = reinterpret_cast<const float4 *>(tab + d.mid + (size_t)(pr0 + 512 * p) * D);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float4 v = src[j];
      Mr[p][2 * j] = pk(v.x, v.y);
      Mr[p][2 * j + 1] = pk(v.z, v.w);
    }
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(barL));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(barM));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // this thread's 4 x 4 block of a chunk: rows ym = 4 w + i, columns yl = 4 lane + j, at
  // float offset blk(i) of a 64-row half of the Lambda1 operand
  auto blk = [&](int i) { return ((4 * w + i) >> 3) * 1152 + lane * 36 + ((4 * w + i) & 7) * 4; };
  // chunk c into hi buffer b (float offset 2 TC_HALF b) and (tid < 68) its M_h1 and r_h2 into
  // sb[b]; each thread copies,
  // and later reads, only its own block
  auto stage = [&](long long c, int b) {
    if (tid < 68) {
      const float *src = (tid < DD / 4) ? tab + d.m1 + (c & mask1) * DD + 4 * tid
                                        : tab + d.r2 + (c >> d.h1) * D + 4 * (tid - DD / 4);
      cp_async16(sb + b * 272 + 4 * tid, src);
    }
    const float *lc = lam + (c << MPS_CHUNK_BITS) + 4 * lane;
#pragma unroll
    for (int i = 0; i < 4; ++i) cp_async16(dyn + 2 * TC_HALF * b + blk(i), lc + (4 * w + i) * 128);
    cp_async_commit();
  };
  auto split = [&](int b, float (&h)[4][4], float (&l)[4][4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 v = *reinterpret_cast<const float4 *>(dyn + 2 * TC_HALF * b + blk(i));
      const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        h[i][j] = tf32_hi(x[j]);
        l[i][j] = x[j] - h[i][j];
      }
    }
  };
  stage(blockIdx.x, 0);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t tw = tmem + ((uint32_t)(32 * (w & 3)) << 16);  // this warp's lane quarter
  unsigned long long P2[2][8];
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int j = 0; j < 8; ++j) P2[p][j] = 0ull;

  // Lambda1 rows of accumulator buffer b into sQ (warps 0..3, lanes = rows)
  auto readout = [&](int b) {
    if (rw) {
      float v[16], u[16];
      tc_ld16(tw + 32 * b, v);  // [lambda_hi; lambda_lo] L_hi, then ... L_lo
      tc_ld16(tw + 32 * b + 16, u);
      float4 *q4 = reinterpret_cast<float4 *>(sQ + (32 * (w & 3) + lane) * 20);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        q4[k] = make_float4(v[4 * k] + u[4 * k], v[4 * k + 1] + u[4 * k + 1], v[4 * k + 2] + u[4 * k + 2],
                            v[4 * k + 3] + u[4 * k + 3]);
    }
  };
  // P and the warp's l_c partial of the chunk whose Lambda1 rows are in sQ and R_c in sr[rb]
  auto update = [&](int rb) {
    unsigned long long L2[2], lc2[8];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int pr = pr0 + 512 * p, ym = pr >> 4, a = pr & 15;
      const float L = sQ[ym * 20 + a] + sQ[(64 + ym) * 20 + a];
      L2[p] = pk(L, L);
    }
    const ulonglong2 *r2 = reinterpret_cast<const ulonglong2 *>(sr + 16 * rb);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const ulonglong2 t = r2[j];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        P2[p][2 * j] = fma2(L2[p], t.x, P2[p][2 * j]);
        P2[p][2 * j + 1] = fma2(L2[p], t.y, P2[p][2 * j + 1]);
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) lc2[j] = fma2(L2[1], Mr[1][j], mul2(L2[0], Mr[0][j]));
    // the 16 values of l_c summed over the warp (transposed halving)
    float v[16];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float2 t = upk(lc2[j]);
      v[2 * j] = t.x;
      v[2 * j + 1] = t.y;
    }
    int cnt = 16;
#pragma unroll
    for (int sh = 16; sh >= 2; sh >>= 1) {
      const int half = cnt / 2;
      const bool hi = (lane & sh) != 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (j < half) {
          const float keep = hi ? v[half + j] : v[j];
          const float send = hi ? v[j] : v[half + j];
          v[j] = keep + __shfl_xor_sync(0xffffffffu, send, sh);
        }
      }
      cnt = half;
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    if ((lane & 1) == 0) {
      const int b = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
      sLc[w * 16 + b] = v[0];
    }
  };
  auto lall_sum = [&](long long cp) {
    if (ls_t >= 0 && ls_t < D) {
      float t = 0.f;
#pragma unroll
      for (int ww = 0; ww < TC_NT / 32; ++ww) t += sLc[ww * 16 + ls_t];
      lall[cp * D + ls_t] = t;
    }
  };
  // the finished mu of one chunk into the FP32 sum (warps 4..7, row yl = 32 (w % 4) + lane each)
  auto add_mu = [&]() {
    if (rw) {
      float v[16], u[16];
      tc_ld16(tw + 64, v);  // lambda^T m_hi and lambda^T m_lo
      tc_ld16(tw + 80, u);
      float4 *row = reinterpret_cast<float4 *>(sMu + (32 * (w & 3) + lane) * 20);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 o = row[j];
        row[j] = make_float4(o.x + (v[4 * j] + u[4 * j]), o.y + (v[4 * j + 1] + u[4 * j + 1]),
                             o.z + (v[4 * j + 2] + u[4 * j + 2]), o.w + (v[4 * j + 3] + u[4 * j + 3]));
      }
    }
  };
  auto flush_mu = [&]() {
    if (rw) {
      const int yl = 32 * (w & 3) + lane;
      float *row = sMu + yl * 20;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        part[a * 128 + yl] += (double)row[a];
        row[a] = 0.f;
      }
    }
  };
  // P into the FP64 partials [pair][b]: each warp's 32 pairs x 16 values go through its own
  // scratch rows (20 floats apart) in the mu copy's region, which is free at every flush
  // point, so that consecutive lanes add into consecutive doubles
  auto flush_p = [&]() {
    float *scr = sAT + w * 32 * 20;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      float4 *row = reinterpret_cast<float4 *>(scr + lane * 20);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 x = upk(P2[p][2 * j]), y = upk(P2[p][2 * j + 1]);
        row[j] = make_float4(x.x, x.y, y.x, y.y);
        P2[p][2 * j] = P2[p][2 * j + 1] = 0ull;
      }
      __syncwarp();
      double *dst = part + 128 * D + (size_t)(pr0 - lane + 512 * p) * D;
#pragma unroll 4
      for (int t = 0; t < 16; ++t) {
        const int e = 32 * t + lane;  // pair e / 16 of the warp, value e % 16
        dst[e] += (double)scr[(e >> 4) * 20 + (e & 15)];
      }
      __syncwarp();
    }
  };

  bool ok = true;
  int since = 0, k = 0, nL = 0, nM = 0;
  long long p = -1, pp = -1;  // the previous chunk; the chunk whose l_c partials sit in sLc
  for (long long c = blockIdx.x; c < chunks; p = c, c += gridDim.x, ++k) {
    const int b = k & 1;
    cp_async_wait<0>();
    __syncthreads();  // B1: sb[b] staged; sLc holds chunk pp's l_c partials
    if (rc_t >= 0 && rc_t < D) {
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j < D; ++j) acc = fmaf(sb[b * 272 + rc_t * D + j], sb[b * 272 + DD + j], acc);
      sr[16 * b + rc_t] = acc;
    }
    if (pp >= 0) lall_sum(pp);
    bool wok = true;
    if (p >= 0) {
      wok = mbar_wait_bounded(barL, (k - 1) & 1);  // Lambda1(p) done: lambda_lo free, its rows ready
      tc_fence_after();
      readout(b ^ 1);
    }
    {
      float h[4][4], l[4][4];
      split(b, h, l);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        *reinterpret_cast<float4 *>(dyn + TC_HALF + blk(i)) = make_float4(l[i][0], l[i][1], l[i][2], l[i][3]);
    }
    if (c + gridDim.x < chunks) stage(c + gridDim.x, b ^ 1);  // hi buffer b ^ 1: Lambda1(p) has read it
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    if (!__syncthreads_and(wok ? 1 : 0)) {  // B2: Lambda1 operands of chunk c in place
      ok = false;
      break;
    }
    tc_fence_after();
    if (issuer) {
      // A: [hi 0; lo] or [lo; hi 1], 16 groups at SBO 4608, K steps of 288 bytes (two core
      // matrices at LBO 144); B: [L_hi | L_lo], N = 32
      const uint64_t a1 = tc_desc(smem_u32(dyn + TC_A1 + b * TC_HALF), 144, 4608);
      const uint64_t lb = tc_desc(smem_u32(dyn + TC_LB), 128, 4096);
#pragma unroll
      for (int s = 0; s < 16; ++s) tc_mma(tmem + 32 * b, a1 + 18 * s, lb + 16 * s, s > 0);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(barL)
                   : "memory");
    }
    ++nL;
    wok = true;
    if (p >= 0) {
      wok = mbar_wait_bounded(barM, (k - 1) & 1);  // mu(p) done: the mu copy and m free
      tc_fence_after();
      add_mu();
    }
    if (since == TC_FLUSH) {
      flush_mu();
      flush_p();
      since = 0;
      __syncthreads();  // every warp's scratch read before the mu copy is written
    }
    {
      float h[4][4], l[4][4];
      split(b, h, l);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int yl = 4 * lane + j;
        const int o = (yl >> 3) * 516 + w * 32 + (yl & 7) * 4;
        *reinterpret_cast<float4 *>(sAT + o) = make_float4(h[0][j], h[1][j], h[2][j], h[3][j]);
        *reinterpret_cast<float4 *>(sAT + 8256 + o) = make_float4(l[0][j], l[1][j], l[2][j], l[3][j]);
      }
      // m(ym)(a) = M(ym)(a, :) R_c for this thread's pairs, split into [m_hi | m_lo]
      const ulonglong2 *r2 = reinterpret_cast<const ulonglong2 *>(sr + 16 * b);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        unsigned long long acc = 0ull;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const ulonglong2 t = r2[j];
          acc = fma2(Mr[q][2 * j], t.x, acc);
          acc = fma2(Mr[q][2 * j + 1], t.y, acc);
        }
        const float2 s2 = upk(acc);
        const float m = s2.x + s2.y, hm = tf32_hi(m);
        const int pr = pr0 + 512 * q, ym = pr >> 4, a = pr & 15;
        const int o = (a >> 3) * 512 + (ym >> 2) * 32 + (a & 7) * 4 + (ym & 3);
        dyn[TC_MB + o] = hm;
        dyn[TC_MB + 1024 + o] = m - hm;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    if (!__syncthreads_and(wok ? 1 : 0)) {  // B3: mu operands of chunk c in place, R_c in sr[b]
      ok = false;
      break;
    }
    tc_fence_after();
    if (issuer) {
      const uint64_t th = tc_desc(smem_u32(sAT), 128, 2064), tl = tc_desc(smem_u32(sAT + 8256), 128, 2064);
      const uint64_t mb = tc_desc(smem_u32(dyn + TC_MB), 128, 2048);
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        tc_mma(tmem + 64, th + 16 * s, mb + 16 * s, s > 0);
        tc_mma(tmem + 64, tl + 16 * s, mb + 16 * s, 1);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(barM)
                   : "memory");
    }
    ++nM;
    ++since;
    if (p >= 0) update(b ^ 1);  // P and l_c of chunk p, while the tensor cores work on chunk c
    pp = p;
  }
  if (ok && k > 0) {
    // the last chunk p: its Lambda1 rows, then P, l_c; then mu and P into the partials
    const int bl = (k - 1) & 1;
    __syncthreads();  // the last update's reads of sQ are done before its rows are replaced
    bool wok = mbar_wait_bounded(barL, (k - 1) & 1);
    tc_fence_after();
    readout(bl);
    wok = mbar_wait_bounded(barM, (k - 1) & 1) && wok;
    tc_fence_after();
    add_mu();
    ok = __syncthreads_and(wok ? 1 : 0) != 0;
    if (ok) {
      if (pp >= 0) lall_sum(pp);
      __syncthreads();
      update(bl);
      __syncthreads();
      lall_sum(p);
      flush_mu();
      flush_p();
    }
  }
  cp_async_wait<0>();
  if (!ok) {
    // a wait ran out: poison this CTA's partials; tensor memory is freed only once both
    // mbarriers report their last commit complete
    for (int i = tid; i < gr.v1; i += TC_NT) part[i] = __longlong_as_double(0x7ff8000000000000LL);
    bool done = true;
    if (nL > 0) done = mbar_wait_bounded(barL, (nL - 1) & 1) && done;
    if (nM > 0) done = mbar_wait_bounded(barM, (nM - 1) & 1) && done;
    ok = __syncthreads_and(done ? 1 : 0) != 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (w == 0 && ok) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

// ----------------------------------------------- bond-16 writer, tensor cores --
// Per 2^13-amplitude chunk the writer's product psi(ym, yl) = sum_a L(yl, a) m(ym, a)
// (L: 128 x 16, m = M_mid R_c: 64 x 16) is one GEMM, 128 x 64 with K = 16.  It runs
// as tcgen05.mma kind::tf32 (M = 128 rows yl, N = 64 columns ym) with the operands
// split into TF32 parts along K: A = [L_hi | L_lo | L_hi], B = [m_hi | m_hi | m_lo]
// (K = 48, six MMAs), which sums L_hi m_hi + L_lo m_hi + L_hi m_lo.  The
// accumulator is double: chunk c - 1 is read out of tensor memory and stored
// (lanes = consecutive yl, 128-byte rows) while chunk c's MMAs run.  m stays on the
// FP32 pipe (thread: one ym, four consecutive a, from the transposed mid matrices in
// shared memory; a 16-byte store per K group of B).  Operand layouts as in the
// gradient pass: K-major, no swizzle, LBO 128 bytes along K, SBO 1536 bytes per
// 8-row group.  The mbarrier waits are bounded; one that runs out stores NaN for
// that chunk, and tensor memory is freed only once the last commits are complete.
constexpr int WT_NT = 512;
constexpr int WT_MLD = 276;                 // floats per ym of the transposed mid matrices (16-byte rows, distinct banks)
constexpr int WT_M = 0;                     // [64 ym][b][a], WT_MLD per ym
constexpr int WT_A = WT_M + 64 * WT_MLD;    // A = [L_hi | L_lo | L_hi]: 16 groups x 1536 bytes
constexpr int WT_B = WT_A + 16 * 384;       // B = [m_hi | m_hi | m_lo], two buffers of 8 groups x 1536 bytes
constexpr int WT_SB = WT_B + 2 * 8 * 384;   // staged M_h1 and r_h2: [2][272]
constexpr int WT_SR = WT_SB + 2 * 272;      // R_c
constexpr int WT_BAR = WT_SR + 16;          // two mbarriers (8 bytes each), tensor-memory address
constexpr size_t WT_SMEM = (size_t)(WT_BAR + 6) * sizeof(float);
// instruction descriptor: FP32 accumulator, TF32 A and B, K-major, M = 128, N = 64
constexpr uint32_t WT_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__global__ void __launch_bounds__(WT_NT, 1) k_mps_write16tc(const PassArgs A) {
  constexpr int D = 16, DD = 256;
  extern __shared__ __align__(16) float dyn[];
  float *sM = dyn + WT_M, *sb = dyn + WT_SB, *sr = dyn + WT_SR;
  // one mbarrier per accumulator buffer: chunk k commits to bar(k % 2) as its (k / 2)-th
  // phase, and every thread waits on it before the next commit to the same barrier (a
  // single barrier could complete two phases before a thread polls it)
  const uint32_t bar0 = smem_u32(dyn + WT_BAR);
  auto bar = [&](int b) { return bar0 + 8 * b; };
  uint32_t *tslot = reinterpret_cast<uint32_t *>(dyn + WT_BAR + 4);
  const MpsDims d = mps_dims(A.n, 4);
  const int job = blockIdx.y, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const float *tab = reinterpret_cast<const float *>(A.in) + (size_t)job * A.in_stride;
  float *out = reinterpret_cast<float *>(A.out) + (size_t)job * A.out_stride;
  const long long chunks = A.tiles;
  const long long mask1 = (1LL << d.h1) - 1;
  const int rc_t = tid - 15 * 32;  // warp 15 lanes 0..15 form R_c
  for (int i = tid; i < 64 * DD; i += WT_NT) {
    const int ym = i / DD, a = (i / D) % D, b = i % D;  // tab: M(ym)(a, b) at (ym D + a) D + b
    sM[ym * WT_MLD + b * D + a] = tab[d.mid + i];
  }
  for (int i = tid; i < 128 * 48; i += WT_NT) {
    const int yl = i / 48, k = i % 48, a = k & 15;
    const float x = tab[d.lo + a * 128 + yl], h = tf32_hi(x);
    dyn[WT_A + (yl >> 3) * 384 + (k >> 2) * 32 + (yl & 7) * 4 + (k & 3)] = (k >> 4) == 1 ? x - h : h;
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar(0)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar(1)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  auto stage = [&](long long c, int b) {
    if (tid < 68) {
      const float *src = (tid < DD / 4) ? tab + d.m1 + (c & mask1) * DD + 4 * tid
                                        : tab + d.r2 + (c >> d.h1) * D + 4 * (tid - DD / 4);
      cp_async16(sb + b * 272 + 4 * tid, src);
    }
    cp_async_commit();
  };
  stage(blockIdx.x, 0);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  // readout: warp w takes tensor-memory lanes 32 (w % 4) .. + 31 (rows yl) and the
  // 16 columns 16 (w / 4) .. + 15 (ym) of an accumulator
  const int sp = w & 3, cb = w >> 2;
  const uint32_t tw = tmem + ((uint32_t)(32 * sp) << 16) + 16 * cb;
  auto store = [&](long long cp, int b, bool good) {
    float v[16];
    tc_ld16(tw + 64 * b, v);
    float *o = out + (cp << MPS_CHUNK_BITS) + (16 * cb) * 128 + 32 * sp + lane;
#pragma unroll
    for (int j = 0; j < 16; ++j) o[j * 128] = good ? v[j] : __int_as_float(0x7fc00000);
  };
  bool ok = true;
  int k = 0, nc = 0;
  long long p = -1;
  for (long long c = blockIdx.x; c < chunks; p = c, c += gridDim.x, ++k) {
    const int b = k & 1;
    cp_async_wait<0>();
    __syncthreads();  // sb[b] staged
    if (rc_t >= 0 && rc_t < D) {
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j < D; ++j) acc = fmaf(sb[b * 272 + rc_t * D + j], sb[b * 272 + DD + j], acc);
      sr[rc_t] = acc;
    }
    if (c + gridDim.x < chunks) stage(c + gridDim.x, b ^ 1);
    __syncthreads();  // R_c in sr
    if (tid < 256) {
      // m(ym)(a) for a = 4 ag .. 4 ag + 3, split into B buffer b (the MMAs that read it,
      // two chunks ago, are complete)
      const int ym = tid & 63, ag = tid >> 6;
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const float4 mv = *reinterpret_cast<const float4 *>(sM + ym * WT_MLD + j * D + 4 * ag);
        const float rj = sr[j];
        acc.x = fmaf(mv.x, rj, acc.x);
        acc.y = fmaf(mv.y, rj, acc.y);
        acc.z = fmaf(mv.z, rj, acc.z);
        acc.w = fmaf(mv.w, rj, acc.w);
      }
      const float4 h = make_float4(tf32_hi(acc.x), tf32_hi(acc.y), tf32_hi(acc.z), tf32_hi(acc.w));
      const float4 l = make_float4(acc.x - h.x, acc.y - h.y, acc.z - h.z, acc.w - h.w);
      float *bb = dyn + WT_B + b * 3072 + (ym >> 3) * 384 + (ym & 7) * 4;
      *reinterpret_cast<float4 *>(bb + ag * 32) = h;
      *reinterpret_cast<float4 *>(bb + (4 + ag) * 32) = h;
      *reinterpret_cast<float4 *>(bb + (8 + ag) * 32) = l;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    if (!__syncthreads_and(ok ? 1 : 0)) break;  // B operand of chunk c in place
    tc_fence_after();
    if (tid == 0) {
      const uint64_t da = tc_desc(smem_u32(dyn + WT_A), 128, 1536);
      const uint64_t db = tc_desc(smem_u32(dyn + WT_B + b * 3072), 128, 1536);
#pragma unroll
      for (int s = 0; s < 6; ++s)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + 64 * b),
            "l"(da + 16 * s), "l"(db + 16 * s), "r"(WT_IDESC), "r"(s > 0 ? 1 : 0));
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar(b))
                   : "memory");
    }
    ++nc;
    if (p >= 0) {
      ok = mbar_wait_bounded(bar(b ^ 1), ((k - 1) >> 1) & 1);  // chunk p's MMAs done
      tc_fence_after();
      store(p, b ^ 1, ok);
    }
    tc_fence_before();
  }
  if (__syncthreads_and(ok ? 1 : 0) && p >= 0) {
    const bool good = mbar_wait_bounded(bar((k - 1) & 1), ((k - 1) >> 1) & 1);  // the last chunk
    tc_fence_after();
    store(p, (k - 1) & 1, good);
  }
  cp_async_wait<0>();
  // tensor memory is freed once the last commit is complete
  tc_fence_before();
  const int n0 = (nc + 1) / 2, n1 = nc / 2;  // commits to bar(0), bar(1)
  const bool done = __syncthreads_and(((n0 == 0 || mbar_wait_bounded(bar(0), (n0 - 1) & 1)) &&
                                       (n1 == 0 || mbar_wait_bounded(bar(1), (n1 - 1) & 1)))
                                          ? 1
                                          : 0) != 0;
  tc_fence_after();
  if (w == 0 && done) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

// High qubits, per (chunk, qubit): block (x, q - 13) takes chunks 256 x .. 256 x + 255
// and qubit q.  Thread c forms u = l_c A_13 .. A_{q-1} and s = A_{q+1} .. A_{n-1} 1
// and adds u dA_q^k s for every layer k <= r; the block's FP64 sums go to its
// partials.  Up to n = 27 (K <= GT_MIN_LEVELS - 1 chunk bits) this is faster than the
// tree below, whose cost is a fixed time per level (measured at n = 27: 82 us
// against 109; at n = 30 the tree takes 0.28 ms against 0.77).
template <int D>
__global__ void __launch_bounds__(256) k_mps_ghigh(const PassArgs A) {
  constexpr int DD = D * D;
  constexpr int ML = DD + 4;  // per-matrix stride: a warp's two matrices (y = 0, 1) on distinct banks
  constexpr int RMAX = 4;
  __shared__ float sA[17 * 2 * ML];
  __shared__ float sdA[(RMAX + 1) * 2 * ML];
  __shared__ double red[8][RMAX + 1];
  const int r = (D == 2) ? 1 : (D == 4 ? 2 : (D == 8 ? 3 : 4));
  const int n = A.n, K = n - MPS_CHUNK_BITS, q = MPS_CHUNK_BITS + blockIdx.y, job = blockIdx.z;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const MpsDims d = mps_dims(n, r);
  const MpsGradRegions gr = mps_grad_regions(n, r);
  const float *tab = reinterpret_cast<const float *>(A.in) + (size_t)job * A.in_stride;
  const float *lall = reinterpret_cast<const float *>(A.lam_in) + (size_t)job * A.lam_stride;
  double *part = A.part + (size_t)job * A.part_stride;
  for (int i = tid; i < K * 2 * DD; i += 256) sA[(i / DD) * ML + i % DD] = tab[d.sites + (long long)MPS_CHUNK_BITS * 2 * DD + i];
  for (int i = tid; i < (r + 1) * 2 * DD; i += 256) {
    const int k = i / (2 * DD), e = i % (2 * DD);
    sdA[(i / DD) * ML + i % DD] = tab[d.dsites + ((long long)k * n + q) * 2 * DD + e];
  }
  __syncthreads();
  const long long c = (long long)blockIdx.x * 256 + tid;
  float val[RMAX + 1] = {0.f, 0.f, 0.f, 0.f, 0.f};
  if (c < A.tiles) {
    float u[D], sv[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      u[a] = lall[c * D + a];
      sv[a] = 1.f;
    }
    for (int j = MPS_CHUNK_BITS; j < q; ++j) {
      const float *M = sA + ((j - MPS_CHUNK_BITS) * 2 + (int)((c >> (j - MPS_CHUNK_BITS)) & 1)) * ML;
      float t[D];
#pragma unroll
      for (int b = 0; b < D; ++b) {
        float acc = 0.f;
#pragma unroll
        for (int a = 0; a < D; ++a) acc = fmaf(u[a], M[a * D + b], acc);
        t[b] = acc;
      }
#pragma unroll
      for (int b = 0; b < D; ++b) u[b] = t[b];
    }
    for (int j = n - 1; j > q; --j) {
      const float *M = sA + ((j - MPS_CHUNK_BITS) * 2 + (int)((c >> (j - MPS_CHUNK_BITS)) & 1)) * ML;
      float t[D];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        float acc = 0.f;
#pragma unroll
        for (int b = 0; b < D; ++b) acc = fmaf(M[a * D + b], sv[b], acc);
        t[a] = acc;
      }
#pragma unroll
      for (int a = 0; a < D; ++a) sv[a] = t[a];
    }
    const int yq = (int)((c >> (q - MPS_CHUNK_BITS)) & 1);
    for (int k = 0; k <= r; ++k) {
      const float *M = sdA + (k * 2 + yq) * ML;
      float acc = 0.f;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        float ra = 0.f;
#pragma unroll
        for (int b = 0; b < D; ++b) ra = fmaf(M[a * D + b], sv[b], ra);
        acc = fmaf(u[a], ra, acc);
      }
      val[k] = acc;
    }
  }
#pragma unroll
  for (int k = 0; k <= RMAX; ++k) {
    float x = val[k];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane == 0) red[w][k] = (double)x;
  }
  __syncthreads();
  if (tid <= r) {
    double t = 0.0;
#pragma unroll
    for (int ww = 0; ww < 8; ++ww) t += red[ww][tid];
    part[gr.part3 + ((long long)(q - MPS_CHUNK_BITS) * (r + 1) + tid) * gr.nb3 + blockIdx.x] = t;
  }
}

// High qubits by a tree over the chunk index bits (level t <-> qubit 13 + t,
// K = n - 13 levels).  With E_t(j) the left environment of the chunks c with
// c >> t == j (l_c A_13 .. A_{12+t}, summed over the low t bits) and R_t(j')
// the right environment A_{14+t} .. A_{n-1} 1 of the bits above t
// (j' = c >> (t + 1)),
//
//   g(k, 13 + t) = sum_j E_t(j) dA^k_{13+t}[j & 1] R_t(j >> 1),
//   E_{t+1}(j)   = E_t(2j) A_{13+t}[0] + E_t(2j + 1) A_{13+t}[1],
//
// which is the per-chunk, per-qubit product of k_mps_ghigh regrouped: D^2 work
// per vector and level instead of D^2 per chunk, qubit and qubit in between.
// Stage 1 (block = 2^B consecutive chunks, B = min(8, K)) runs levels 0..B-1 inside
// the block from the right environment of its own index bits and leaves E_B in
// the block's first chunk vector; stage 2 (one block per job) runs levels B..K-1
// over those.  Each (vector, layer) term is formed in FP32 and summed in FP64 in
// a fixed order; the sums go to the same partial slots k_mps_ghigh fills.
constexpr int GT_NT = 256;
constexpr int GT_BLOCK_BITS = 8;  // stage 1: 2^8 chunks per block, one block per partial slot
constexpr int GT_MIN_LEVELS = 15; // the tree from n = 28 (15 chunk bits); per (chunk, qubit) below
// (stage 2 takes the other n - 21 <= 9 levels: at most 2^9 vectors, 150 KB at D = 16)
template <int D>
__global__ void __launch_bounds__(GT_NT) k_mps_gtree(const PassArgs A, int t0, int L, int sh) {
  constexpr int DD = D * D;
  constexpr int RMAX = 4;
  const int r = (D == 2) ? 1 : (D == 4 ? 2 : (D == 8 ? 3 : 4));
  const int n = A.n, K = n - MPS_CHUNK_BITS, job = blockIdx.y, tid = threadIdx.x;
  const long long blk = blockIdx.x;
  const int NV = 1 << L;
  const MpsDims d = mps_dims(n, r);
  const MpsGradRegions gr = mps_grad_regions(n, r);
  const float *tab = reinterpret_cast<const float *>(A.in) + (size_t)job * A.in_stride;
  // the chunk vectors sit in this step's partial region (writable): stage 1 leaves each
  // block's E_B there for stage 2
  float *lall = const_cast<float *>(reinterpret_cast<const float *>(A.lam_in)) + (size_t)job * A.lam_stride;
  double *part = A.part + (size_t)job * A.part_stride;
  extern __shared__ __align__(16) float gdyn[];
  // shared memory sized by this stage's NV vectors (gtree_smem)
  float *sA = gdyn;              // A_{13+t}[y] for t < K: [K][2][DD]
  float *sE = sA + K * 2 * DD;   // E ping-pong: [2][NV][D]
  float *sR = sE + 2 * NV * D;   // R of every level: level lt's 2^(L-1-lt) vectors from vector 2^(L-1-lt) - 1
  float *sd = sR + NV * D;       // dA^k_q[y]: [RMAX + 1][2][DD]
  double *sv = reinterpret_cast<double *>(sd + (RMAX + 1) * 2 * DD);  // terms [RMAX + 1][NV / 2]
  __shared__ float sRt[D];
  __shared__ double sg[RMAX + 1];
  for (int i = tid; i < K * 2 * DD; i += GT_NT) sA[i] = tab[d.sites + (long long)MPS_CHUNK_BITS * 2 * DD + i];
  for (int i = tid; i < NV * D; i += GT_NT) {
    const int v = i / D, a = i % D;
    sE[i] = lall[(((blk << L) + v) << sh) * D + a];
  }
  __syncthreads();
  // the right environment of the bits above this block: levels t0 + L .. K - 1
  if (tid < 32) {
    float x = (tid < D) ? 1.f : 0.f;
    for (int t = K - 1; t >= t0 + L; --t) {
      const int y = (int)((blk >> (t - t0 - L)) & 1);
      const float *M = sA + (t * 2 + y) * DD;
      float acc = 0.f;
      if (tid < D) {
#pragma unroll
        for (int b = 0; b < D; ++b) acc = fmaf(M[tid * D + b], __shfl_sync(0xffffffffu, x, b), acc);
      } else {
#pragma unroll
        for (int b = 0; b < D; ++b) (void)__shfl_sync(0xffffffffu, x, b);
      }
      x = acc;
    }
    if (tid < D) sRt[tid] = x;
  }
  __syncthreads();
  // R of level lt (local) holds 2^(L-1-lt) vectors at sR + (2^(L-1-lt) - 1) D: level L-1 is
  // R_top, level lt from level lt + 1 through A_{14+t0+lt}
  if (tid < D) sR[tid] = sRt[tid];
  __syncthreads();
  for (int lt = L - 2; lt >= 0; --lt) {
    const int cnt = 1 << (L - 1 - lt), t = t0 + lt;
    float *dst = sR + (cnt - 1) * D;
    const float *src = sR + (cnt / 2 - 1) * D;
    for (int i = tid; i < cnt * D; i += GT_NT) {
      const int jp = i / D, a = i % D;
      const float *M = sA + ((t + 1) * 2 + (jp & 1)) * DD;
      const float *s = src + (jp >> 1) * D;
      float acc = 0.f;
#pragma unroll
      for (int b = 0; b < D; ++b) acc = fmaf(M[a * D + b], s[b], acc);
      dst[i] = acc;
    }
    __syncthreads();
  }
  int cur = 0;
  for (int lt = 0; lt < L; ++lt) {
    const int t = t0 + lt, q = MPS_CHUNK_BITS + t, nv = 1 << (L - lt);
    for (int i = tid; i < (r + 1) * 2 * DD; i += GT_NT) {
      const int k = i / (2 * DD), e = i % (2 * DD);
      sd[i] = tab[d.dsites + ((long long)k * n + q) * 2 * DD + e];
    }
    __syncthreads();
    const float *E = sE + cur * NV * D;
    const float *R = sR + (nv / 2 - 1) * D;
    // term (k, j) = E(j) dA^k[j & 1] R(j >> 1); pairs of vectors j = 2 i, 2 i + 1 share R
    for (int i = tid; i < (r + 1) * (nv / 2); i += GT_NT) {
      const int k = i / (nv / 2), jj = i % (nv / 2);
      const float *Rv = R + jj * D;
      double tsum = 0.0;
#pragma unroll
      for (int y = 0; y < 2; ++y) {
        const float *M = sd + (k * 2 + y) * DD;
        const float *Ev = E + (2 * jj + y) * D;
        float acc = 0.f;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          float ra = 0.f;
#pragma unroll
          for (int b = 0; b < D; ++b) ra = fmaf(M[a * D + b], Rv[b], ra);
          acc = fmaf(Ev[a], ra, acc);
        }
        tsum += (double)acc;
      }
      sv[k * (NV / 2) + jj] = tsum;
    }
    // E of the next level
    float *En = sE + (cur ^ 1) * NV * D;
    for (int i = tid; i < (nv / 2) * D; i += GT_NT) {
      const int j = i / D, b = i % D;
      const float *M0 = sA + (t * 2) * DD, *M1 = M0 + DD;
      const float *E0 = E + (2 * j) * D, *E1 = E0 + D;
      float acc = 0.f;
#pragma unroll
      for (int a = 0; a < D; ++a) acc = fmaf(E1[a], M1[a * D + b], fmaf(E0[a], M0[a * D + b], acc));
      En[i] = acc;
    }
    __syncthreads();
    if (tid <= r) {
      double s = 0.0;
      for (int jj = 0; jj < nv / 2; ++jj) s += sv[tid * (NV / 2) + jj];
      sg[tid] = s;
    }
    __syncthreads();
    if (tid <= r) part[gr.part3 + ((long long)t * (r + 1) + tid) * gr.nb3 + (t0 == 0 ? blk : 0)] = sg[tid];
    cur ^= 1;
  }
  if (t0 == 0) {
    // E_L of this block into its first chunk vector (all of the block's reads are done);
    // the levels above this stage start at zero in this block's slot, and slots no
    // block of this stage owns are zero
    if (tid < D) lall[((blk << L) << sh) * D + tid] = sE[cur * NV * D + tid];
    for (int i = tid; i < (K - L) * (r + 1); i += GT_NT)
      part[gr.part3 + ((long long)(L + i / (r + 1)) * (r + 1) + i % (r + 1)) * gr.nb3 + blk] = 0.0;
    for (long long s = blk + gridDim.x; s < gr.nb3; s += gridDim.x)
      for (int i = tid; i < K * (r + 1); i += GT_NT) part[gr.part3 + (long long)i * gr.nb3 + s] = 0.0;
  }
}

// Fixed-order FP64 sums: value v < v1 over the CTAs of k_mps_grad, the rest
// (high qubit, layer) over the slots of k_mps_ghigh or k_mps_gtree.
__global__ void __launch_bounds__(128) k_mps_gred(const PassArgs A) {
  const int r = A.layer, job = blockIdx.y;
  const MpsGradRegions gr = mps_grad_regions(A.n, r);
  const long long v = (long long)blockIdx.x * 128 + threadIdx.x;
  if (v >= gr.v1 + gr.k * (r + 1)) return;
  const double *p = A.part + (size_t)job * A.part_stride;
  double t = 0.0;
  if (v < gr.v1) {
    for (long long c = 0; c < gr.gc; ++c) t += p[gr.part1 + c * gr.v1 + v];
  } else {
    const long long i = v - gr.v1;
    for (long long b = 0; b < gr.nb3; ++b) t += p[gr.part3 + i * gr.nb3 + b];
  }
  A.part[(size_t)job * A.part_stride + gr.red + v] = t;
}

// Gradients of qubits 0..12 (block q) from the summed mu and P, and the high
// qubits' sums copied (block 13).  Qubit q in 0..6: thread y (a pattern of
// qubits 0..6) forms x = e_0 A_0 .. A_{q-1} and s = A_{q+1} .. A_6 mu(y);
// qubit q in 7..12: thread (y, a) (a pattern of qubits 7..12 and a row) forms
// x = e_a A_7 .. A_{q-1} and s = A_{q+1} .. A_12 P(y)(a, :); each adds
// x dA_q^k s, summed in FP64.
template <int D>
__global__ void __launch_bounds__(256) k_mps_genv(const PassArgs A) {
  constexpr int DD = D * D;
  constexpr int RMAX = 4;
  __shared__ double red[8][RMAX + 1];
  const int r = (D == 2) ? 1 : (D == 4 ? 2 : (D == 8 ? 3 : 4));
  const int n = A.n, q = blockIdx.x, job = blockIdx.y, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const MpsDims d = mps_dims(n, r);
  const MpsGradRegions gr = mps_grad_regions(n, r);
  const float *tab = reinterpret_cast<const float *>(A.in) + (size_t)job * A.in_stride;
  const double *sums = A.part + (size_t)job * A.part_stride + gr.red;
  double *fin = A.part + (size_t)job * A.part_stride + gr.fin;
  if (q == MPS_CHUNK_BITS) {
    for (int i = tid; i < gr.k * (r + 1); i += 256) {
      const int qq = MPS_CHUNK_BITS + i / (r + 1), k = i % (r + 1);
      fin[(long long)k * n + qq] = 2.0 * sums[gr.v1 + i];
    }
    return;
  }
  auto site = [&](int j, int y) { return tab + d.sites + ((long long)j * 2 + y) * DD; };
  const bool lo = q < 7;
  const int nitems = lo ? 128 : 64 * D;
  double acc[RMAX + 1] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int it = tid; it < nitems; it += 256) {
    const int pat = lo ? it : it / D, a0 = lo ? 0 : it % D;
    const int q0 = lo ? 0 : 7, q1 = lo ? 7 : 13;
    float x[D], sv[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      x[a] = (a == a0) ? 1.f : 0.f;
      sv[a] = lo ? (float)sums[(long long)a * 128 + pat] : (float)sums[128 * D + ((long long)pat * D + a0) * D + a];
    }
    for (int j = q0; j < q; ++j) {
      const float *M = site(j, (pat >> (j - q0)) & 1);
      float t[D];
#pragma unroll
      for (int b = 0; b < D; ++b) {
        float s = 0.f;
#pragma unroll
        for (int a = 0; a < D; ++a) s = fmaf(x[a], M[a * D + b], s);
        t[b] = s;
      }
#pragma unroll
      for (int b = 0; b < D; ++b) x[b] = t[b];
    }
    for (int j = q1 - 1; j > q; --j) {
      const float *M = site(j, (pat >> (j - q0)) & 1);
      float t[D];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        float s = 0.f;
#pragma unroll
        for (int b = 0; b < D; ++b) s = fmaf(M[a * D + b], sv[b], s);
        t[a] = s;
      }
#pragma unroll
      for (int a = 0; a < D; ++a) sv[a] = t[a];
    }
    const int yq = (pat >> (q - q0)) & 1;
    for (int k = 0; k <= r; ++k) {
      const float *M = tab + d.dsites + (((long long)k * n + q) * 2 + yq) * DD;
      double s = 0.0;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        float ra = 0.f;
#pragma unroll
        for (int b = 0; b < D; ++b) ra = fmaf(M[a * D + b], sv[b], ra);
        s += (double)x[a] * (double)ra;
      }
      acc[k] += s;
    }
  }
#pragma unroll
  for (int k = 0; k <= RMAX; ++k) {
    double x = acc[k];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane == 0) red[w][k] = x;
  }
  __syncthreads();
  if (tid <= r) {
    double t = 0.0;
#pragma unroll
    for (int ww = 0; ww < 8; ++ww) t += red[ww][tid];
    fin[(long long)tid * n + q] = 2.0 * t;
  }
}

template <int D>
cudaError_t launch_mps_grad_d(const PassArgs &A, int jobs, cudaStream_t s) {
  const MpsGradRegions gr = mps_grad_regions(A.n, A.layer);
  switch (A.kind) {
    case K_MPS_GRAD: {
      if constexpr (D >= 16) {
        if (A.flags & F_MPS_TC) {
          cudaFuncSetAttribute(k_mps_grad16tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
          k_mps_grad16tc<<<dim3((unsigned)gr.gc, (unsigned)jobs), TC_NT, TC_SMEM, s>>>(A);
          break;
        }
        const size_t smem = (size_t)(2 * 64 * LAM_LD + 64 * D * G16_RS + 128 * D + 4 * 64 * G16_RS) * sizeof(float);
        cudaFuncSetAttribute(k_mps_grad16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_mps_grad16<<<dim3((unsigned)gr.gc, (unsigned)jobs), G16_NT, smem, s>>>(A);
      } else {
        const size_t smem = (size_t)(2 * 64 * LAM_LD + 64 * (D * D + D) + 128 * D + 4 * 64 * D) * sizeof(float);
        cudaFuncSetAttribute(k_mps_grad<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_mps_grad<D><<<dim3((unsigned)gr.gc, (unsigned)jobs), GR_NT, smem, s>>>(A);
      }
      break;
    }
    case K_MPS_GHIGH: {
      const int K = A.n - MPS_CHUNK_BITS, B = K < GT_BLOCK_BITS ? K : GT_BLOCK_BITS;
      if (K < GT_MIN_LEVELS) {
        k_mps_ghigh<D><<<dim3((unsigned)gr.nb3, (unsigned)gr.k, (unsigned)jobs), 256, 0, s>>>(A);
        break;
      }
      // shared memory of a stage with NV = 2^L vectors
      auto gtree_smem = [&](int L) {
        const size_t nv = (size_t)1 << L;
        return (size_t)(K * 2 * D * D + 3 * nv * D + 10 * D * D) * sizeof(float) + 5 * (nv / 2) * sizeof(double);
      };
      cudaFuncSetAttribute(k_mps_gtree<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)gtree_smem(K > B ? (K - B > B ? K - B : B) : B));
      k_mps_gtree<D><<<dim3((unsigned)(1LL << (K - B)), (unsigned)jobs), GT_NT, gtree_smem(B), s>>>(A, 0, B, 0);
      if (K > B) k_mps_gtree<D><<<dim3(1, (unsigned)jobs), GT_NT, gtree_smem(K - B), s>>>(A, B, K - B, B);
      break;
    }
    case K_MPS_GRED:
      k_mps_gred<<<dim3((unsigned)((gr.v1 + gr.k * (A.layer + 1) + 127) / 128), (unsigned)jobs), 128, 0, s>>>(A);
      break;
    default:  // K_MPS_GENV
      k_mps_genv<D><<<dim3(MPS_CHUNK_BITS + 1, (unsigned)jobs), 256, 0, s>>>(A);
      break;
  }
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_mps_d(const PassArgs &A, int jobs, cudaStream_t s) {
  if (A.kind >= K_MPS_GRAD) return launch_mps_grad_d<D>(A, jobs, s);
  if (A.kind == K_MPS_TAB) {
    const MpsDims d = mps_dims(A.n, A.layer);
    const MpsItems its = mps_items(d);
    long long blocks = (its.total + TAB_NT - 1) / TAB_NT;
    if (A.flags & F_MPS_SITES) blocks += ((long long)A.n * 2 * D * D * (A.layer + 2) + TAB_NT - 1) / TAB_NT;
    const dim3 grid((unsigned)blocks, (unsigned)jobs);
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
  if constexpr (D >= 16) {
    if (A.flags & F_MPS_TC) {
      const long long ctas = num_sms_cached();
      cudaFuncSetAttribute(k_mps_write16tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WT_SMEM);
      k_mps_write16tc<<<dim3((unsigned)(A.tiles < ctas ? A.tiles : ctas), (unsigned)jobs), WT_NT, WT_SMEM, s>>>(A);
      return cudaGetLastError();
    }
  }
  const long long cap = (long long)num_sms_cached() * (D >= 16 ? 2 : 4);
  const dim3 grid((unsigned)(A.tiles < cap ? A.tiles : cap), (unsigned)jobs);
  const size_t smem = (size_t)64 * (D * D + D) * sizeof(float);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_mps_write<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_mps_write<D><<<grid, WR_NT, smem, s>>>(A);
  return cudaGetLastError();
}

}  // namespace

int mps_step_kernels(const PassArgs &A) {
  if (A.kind == K_MPS_GHIGH) return (A.n - MPS_CHUNK_BITS >= GT_MIN_LEVELS) ? 2 : 1;
  return 1;
}

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
