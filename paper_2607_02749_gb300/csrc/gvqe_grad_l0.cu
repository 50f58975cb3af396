// gvqe_grad_l0.cu -- the layer-0 gradient pass.
//
// Once the adjoint sweep has carried lambda back through every layer above
// the first RY layer, the gradients of that layer (dE/dtheta of Eq. 13 for the
// first RY layer of Section IV-B) follow from lambda_0 and the analytic
// product state psi_0(x) = prod_q f_q(x_q):
//
//   g_{0,q} = sum_x lambda_0(x) d_q(x_q) prod_{q' != q} f_q'(x_q')
//   f_q(0) = cos(t_q/2), f_q(1) = sin(t_q/2), d_q(0) = -sin(t_q/2), d_q(1) = cos(t_q/2)
//
// (the 1/2 of d cos(t/2)/dt and the 2 of dE = 2 <lambda|dpsi> cancel).
//
// Every warp works alone -- no block barrier after the set-up -- on "groups"
// of 2^(10+mb) amplitudes, bits of x = [group | m (mb bits) | kk (3) | lane (5) | j (2)]:
//   j      two bits held in one 16-byte load of four consecutive amplitudes,
//   kk     eight such loads per lane and chunk of 1024 amplitudes,
//   lane   the warp lane,
//   m      the chunks of one group, weighted by a tabulated factor H(m),
//   group  the factor F_q(group) of the remaining qubits, one per lane q.
// Per chunk a lane contracts its 32 amplitudes with the factors of bits
// 0, 1, 7, 8, 9 as a tree (the value and the five one-bit derivatives share
// their partial contractions); per group one transposed warp reduction brings
// the sum for qubit q to lane q, which multiplies it by F_q(group) and adds it
// to an FP64 accumulator.  The next chunk's loads are issued before the
// current chunk is contracted (two register buffers).
#include "gvqe_engine.cuh"

namespace gvqe {

int num_sms_cached();

namespace {

constexpr int GL_NT = 256;
constexpr int GL_NW = GL_NT / 32;

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

// four consecutive amplitudes starting at a 16-byte aligned element
__device__ __forceinline__ void ld_quad(const float *p, float (&v)[4]) {
  const float4 q = __ldcg(reinterpret_cast<const float4 *>(p));
  v[0] = q.x;
  v[1] = q.y;
  v[2] = q.z;
  v[3] = q.w;
}
__device__ __forceinline__ void ld_quad(const double *p, double (&v)[4]) {
  const double2 a = __ldcg(reinterpret_cast<const double2 *>(p));
  const double2 b = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}

// Sum over the warp of 16 per-lane values at once: after the call lanes 2i
// and 2i+1 hold the warp sum of value i.  Each halving step keeps the half of
// the values selected by one lane bit and sends the other half to the partner.
template <typename T>
__device__ __forceinline__ T reduce16(const T (&v)[16], int lane) {
  T u8[8], u4[4], u2[2];
  {
    const bool b = (lane >> 4) & 1;
#pragma unroll
    for (int j = 0; j < 8; ++j) u8[j] = (b ? v[8 + j] : v[j]) + __shfl_xor_sync(0xffffffffu, b ? v[j] : v[8 + j], 16);
  }
  {
    const bool b = (lane >> 3) & 1;
#pragma unroll
    for (int j = 0; j < 4; ++j) u4[j] = (b ? u8[4 + j] : u8[j]) + __shfl_xor_sync(0xffffffffu, b ? u8[j] : u8[4 + j], 8);
  }
  {
    const bool b = (lane >> 2) & 1;
#pragma unroll
    for (int j = 0; j < 2; ++j) u2[j] = (b ? u4[2 + j] : u4[j]) + __shfl_xor_sync(0xffffffffu, b ? u4[j] : u4[2 + j], 4);
  }
  const bool b = (lane >> 1) & 1;
  T r = (b ? u2[1] : u2[0]) + __shfl_xor_sync(0xffffffffu, b ? u2[0] : u2[1], 2);
  return r + __shfl_xor_sync(0xffffffffu, r, 1);
}

// Reduction slot of qubit q: 0 the plain sum (qubits of the group factor),
// 1..5 the register-bit derivatives (qubits 0, 1, 7, 8, 9), 6..10 the lane-bit
// derivatives (qubits 2..6), 12..14 the chunk-bit derivatives (qubits 10..10+mb-1).
__device__ __forceinline__ int slot_of(int q, int mb) {
  if (q == 0) return 1;
  if (q == 1) return 2;
  if (q <= 6) return 6 + (q - 2);
  if (q <= 9) return 3 + (q - 7);
  if (q < 10 + mb) return 12 + (q - 10);
  return 0;
}

template <typename T, bool INIT>
__global__ void __launch_bounds__(GL_NT, sizeof(T) == 4 ? 2 : 1) k_grad_l0w(const PassArgs A) {
  using T2 = typename V2<T>::type;
  __shared__ T2 l0cs[32];
  __shared__ T Ht[4][8];  // [0][m] = H(m); [1+r][m] = H(m) with the factor of qubit 10+r differentiated

  const int job = blockIdx.y;
  if (A.minlayer != nullptr && !(A.flags & F_ENERGY) && A.minlayer[A.job0 + job] > 0) return;
  const int tid = threadIdx.x, lane = tid & 31;
  const int n = A.n, mb = A.c;
  const T2 *cs = reinterpret_cast<const T2 *>(A.cs) + (size_t)(A.job0 + job) * A.P;
  if (tid < n) l0cs[tid] = cs[tid];
  __syncthreads();
  if (tid < 32) {
    const int r = tid >> 3, m = tid & 7;
    T h = T(0);
    if (m < (1 << mb) && (r == 0 || r - 1 < mb)) {
      h = T(1);
      for (int i = 0; i < mb; ++i) {
        const T2 c = l0cs[10 + i];
        const int b = (m >> i) & 1;
        h *= (r == 1 + i) ? (b ? c.x : -c.y) : (b ? c.y : c.x);
      }
    }
    Ht[r][m] = h;
  }
  __syncthreads();

  const long long W = A.tiles;  // warps (= partials per qubit) per job
  const long long gw = (long long)blockIdx.x * GL_NW + (tid >> 5);
  if (gw >= W) return;
  const int hb = 10 + mb;                     // first qubit of the group factor
  const long long G = 1LL << (n - hb);        // groups per job
  const long long ngroups = (G - gw + W - 1) / W;
  const int M = 1 << mb;
  const long long S = ngroups * M;  // chunks of this warp

  // factors of the register bits 0, 1, 7, 8, 9
  T c0, s0, c1, s1, c7, s7, c8, s8, c9, s9;
  c0 = l0cs[0].x, s0 = l0cs[0].y, c1 = l0cs[1].x, s1 = l0cs[1].y;
  c7 = l0cs[7].x, s7 = l0cs[7].y, c8 = l0cs[8].x, s8 = l0cs[8].y, c9 = l0cs[9].x, s9 = l0cs[9].y;
  // lane bits 2..6
  T lane_f = T(1), lane_d[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const T2 c = l0cs[2 + j];
    lane_f *= ((lane >> j) & 1) ? c.y : c.x;
  }
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    T g = T(1);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const T2 c = l0cs[2 + i];
      const int b = (lane >> i) & 1;
      g *= (i == j) ? (b ? c.x : -c.y) : (b ? c.y : c.x);
    }
    lane_d[j] = g;
  }
  // product-state factors of bits (0,1) and (7,8,9), for lambda = E * psi_0
  T Pj[4], Pk[8];
  if (INIT) {
#pragma unroll
    for (int j = 0; j < 4; ++j) Pj[j] = ((j & 1) ? s0 : c0) * ((j & 2) ? s1 : c1);
#pragma unroll
    for (int k = 0; k < 8; ++k) Pk[k] = ((k & 1) ? s7 : c7) * ((k & 2) ? s8 : c8) * ((k & 4) ? s9 : c9);
  }
  const int src = 2 * slot_of(lane, mb);

  const T *base = INIT ? reinterpret_cast<const T *>(A.table) + (size_t)job * A.table_stride
                       : reinterpret_cast<const T *>(A.lam_in) + (size_t)job * A.lam_stride;
  const int lofs = 4 * lane;
  auto chunk_ptr = [&](long long s) -> const T * {
    const long long g = gw + (s >> mb) * W;
    const long long x0 = ((g << mb) + (s & (M - 1))) << 10;
    return base + x0 + lofs;
  };

  T acc_S = T(0), acc_j[5] = {T(0), T(0), T(0), T(0), T(0)}, acc_h[3] = {T(0), T(0), T(0)}, eacc = T(0);
  T Fq = T(1), Fpure = T(1);
  double acc_g = 0.0, acc_e = 0.0;

  auto step = [&](T (&v)[8][4], long long s) {
    const int m = (int)(s & (M - 1));
    if (m == 0) {  // group factor of this lane's qubit
      const long long g = gw + (s >> mb) * W;
      T f = T(1);
      for (int i = hb; i < n; ++i) {
        const T2 c = l0cs[i];
        const int b = (int)((g >> (i - hb)) & 1);
        f *= (i == lane) ? (b ? c.x : -c.y) : (b ? c.y : c.x);
      }
      Fq = f;
      if (INIT) Fpure = __shfl_sync(0xffffffffu, f, 0);
    }
    const T H = Ht[0][m];
    if (INIT) {
      const T pb = lane_f * H * Fpure;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const T pk = pb * Pk[k];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const T psi = pk * Pj[j];
          const T lam = v[k][j] * psi;
          eacc += psi * lam;
          v[k][j] = lam;
        }
      }
    }
    // bit 0
    T a[8][2], b[8][2];
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        a[k][h] = c0 * v[k][2 * h] + s0 * v[k][2 * h + 1];
        b[k][h] = c0 * v[k][2 * h + 1] - s0 * v[k][2 * h];
      }
    // bit 1
    T aa[8], ab[8], ba[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      aa[k] = c1 * a[k][0] + s1 * a[k][1];
      ab[k] = c1 * a[k][1] - s1 * a[k][0];
      ba[k] = c1 * b[k][0] + s1 * b[k][1];
    }
    // bits 7, 8, 9
    auto contract3 = [&](const T (&u)[8]) -> T {
      T w4[4], w2[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) w4[i] = c7 * u[2 * i] + s7 * u[2 * i + 1];
#pragma unroll
      for (int i = 0; i < 2; ++i) w2[i] = c8 * w4[2 * i] + s8 * w4[2 * i + 1];
      return c9 * w2[0] + s9 * w2[1];
    };
    const T S0 = contract3(ba);
    const T S1 = contract3(ab);
    T p4[4], pd4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      p4[i] = c7 * aa[2 * i] + s7 * aa[2 * i + 1];
      pd4[i] = c7 * aa[2 * i + 1] - s7 * aa[2 * i];
    }
    T q2[2], qd2[2], pd2[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      q2[i] = c8 * p4[2 * i] + s8 * p4[2 * i + 1];
      qd2[i] = c8 * p4[2 * i + 1] - s8 * p4[2 * i];
      pd2[i] = c8 * pd4[2 * i] + s8 * pd4[2 * i + 1];
    }
    const T S7 = c9 * pd2[0] + s9 * pd2[1];
    const T S8 = c9 * qd2[0] + s9 * qd2[1];
    const T Sv = c9 * q2[0] + s9 * q2[1];
    const T S9 = c9 * q2[1] - s9 * q2[0];

    acc_S += H * Sv;
    acc_j[0] += H * S0;
    acc_j[1] += H * S1;
    acc_j[2] += H * S7;
    acc_j[3] += H * S8;
    acc_j[4] += H * S9;
#pragma unroll
    for (int r = 0; r < 3; ++r) acc_h[r] += Ht[1 + r][m] * Sv;

    if (m == M - 1) {  // group complete: warp sums, qubit q to lane q
      T vals[16];
      vals[0] = lane_f * acc_S;
#pragma unroll
      for (int j = 0; j < 5; ++j) vals[1 + j] = lane_f * acc_j[j];
#pragma unroll
      for (int j = 0; j < 5; ++j) vals[6 + j] = lane_d[j] * acc_S;
      vals[11] = eacc;
#pragma unroll
      for (int r = 0; r < 3; ++r) vals[12 + r] = lane_f * acc_h[r];
      vals[15] = T(0);
      const T r = reduce16(vals, lane);
      const T val = __shfl_sync(0xffffffffu, r, src);
      acc_g += (double)Fq * (double)val;
      if (INIT) acc_e += (double)__shfl_sync(0xffffffffu, r, 22);
      acc_S = T(0);
#pragma unroll
      for (int j = 0; j < 5; ++j) acc_j[j] = T(0);
#pragma unroll
      for (int j = 0; j < 3; ++j) acc_h[j] = T(0);
      eacc = T(0);
    }
  };

  T va[8][4], vb[8][4];
  auto load = [&](T (&v)[8][4], long long s) {
    const T *p = chunk_ptr(s);
#pragma unroll
    for (int k = 0; k < 8; ++k) ld_quad(p + 128 * k, v[k]);
  };
  load(va, 0);
  for (long long s = 0; s < S; s += 2) {
    if (s + 1 < S) load(vb, s + 1);
    step(va, s);
    if (s + 2 < S) load(va, s + 2);
    if (s + 1 < S) step(vb, s + 1);
  }

  double *part = A.part + (size_t)job * A.part_stride;
  if (lane < n) part[(size_t)lane * W + gw] = acc_g;
  if (INIT && lane == 0) A.epart[(size_t)job * A.part_stride + gw] = acc_e;
}

template <typename T>
cudaError_t launch_typed(const PassArgs &A, int jobs, cudaStream_t s) {
  const dim3 grid((unsigned)((A.tiles + GL_NW - 1) / GL_NW), (unsigned)jobs);
  if (A.flags & F_LAMBDA_INIT)
    k_grad_l0w<T, true><<<grid, GL_NT, 0, s>>>(A);
  else
    k_grad_l0w<T, false><<<grid, GL_NT, 0, s>>>(A);
  return cudaGetLastError();
}

}  // namespace

void grad_l0_layout(int n, int prec, int *mb, long long *slots) {
  int b = n - 22;  // fold chunk bits into a group only while 2^11 groups remain
  if (b < 0) b = 0;
  if (b > 3) b = 3;
  if (b > n - 10) b = n - 10;
  const long long groups = 1LL << (n - 10 - b);
  long long w = (long long)num_sms_cached() * (prec ? 1 : 2) * GL_NW;
  if (w > groups) w = groups;
  *mb = b;
  *slots = w;
}

cudaError_t launch_grad_l0(int prec, const PassArgs &A, int jobs, cudaStream_t s) {
  if (A.n < 10 || A.c < 0 || A.c > 3 || A.c > A.n - 10 || A.tiles < 1 || A.tiles > (1LL << (A.n - 10 - A.c)))
    return cudaErrorInvalidValue;
  return prec ? launch_typed<double>(A, jobs, s) : launch_typed<float>(A, jobs, s);
}

}  // namespace gvqe
