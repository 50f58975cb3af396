// gvqe_engine.cuh -- launch descriptors shared by the host planner and the kernels.
//
// The state vector of n qubits is a real array of 2^n amplitudes (float or
// double): the RY+CX ansatz of Section IV-B maps |0> to a real vector (RY is a
// real rotation, CX a permutation), so the imaginary part is identically zero
// and is not stored.
//
// Work is organised in "tile passes".  A tile is 2^tb amplitudes whose index
// bits are tile-local bits [0, c) -> global bits [0, c) (contiguous runs that
// keep global accesses coalesced) and tile-local bits [c, tb) -> global bits
// [a, a + tb - c), or, split in two runs, [c, c + k1) -> [a, a + k1) and
// [c + k1, tb) -> [a + k1 + gap, a + gap + tb - c) (gap = 0: one run).  The
// remaining global bits enumerate the tiles.  A pass applies the RY gates of
// one layer on the qubits of its gate bits while the tile sits on chip; an RY
// layer on n qubits takes one pass over bits [0, tb) plus passes over the
// higher qubits.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gvqe {

enum PassKind : int {
  K_FWD = 0,        // forward: RY(theta) on the gate bits of one layer
  K_BWD = 1,        // adjoint: gradients of the gate bits, then RY(-theta) on lambda
  K_GRAD_L0 = 2,    // layer-0 gradients against the analytic product state
  K_LAMBDA_XY = 3,  // lambda = H psi with X-mask groups; energy
  K_WHT = 4,        // unnormalised Walsh-Hadamard butterflies (diagonal table build)
  K_MPS = 5,        // a leading layer's state written in closed form (gvqe_mps.cu)
  K_MPS_TAB = 6,    // the contracted site-tensor tables K_MPS reads
  K_MPS_GRAD = 7,   // gradients of the closed-form layers: one pass over lambda (environments)
  K_MPS_GHIGH = 8,  // ... the qubits above the 2^13-amplitude chunk, per chunk and qubit
  K_MPS_GRED = 9,   // ... fixed-order FP64 sums of the per-CTA partials
  K_MPS_GENV = 10,  // ... the qubits inside the chunk, from the summed environments
};

enum LoadMode : int {
  LD_PLAIN = 0,      // v = in[y]
  LD_GATHER = 1,     // v = in[A^-1 y]: the linear CX chain applied on the fly
  LD_L0_GATHER = 2,  // v = psi_0(A^-1 y): analytic layer-0 product state through the CX chain
  LD_L0 = 3,         // v = psi_0(y)
  LD_ZERO = 4,       // v = |0...0>: 1 at index 0, else 0 (the complex path's layer 0)
};

// Entanglers (Section IV-B; Table 2 adds reverse linear, pairwise and SCA).  As
// a map of basis indices each entangler layer is GF(2)-linear, y = A x; passes
// need x = A^-1 y (gather for psi, scatter for lambda):
//   ENT_LINEAR          CX(0,1)..CX(n-2,n-1): y = prefix XOR of x,  x = y ^ (y << 1)
//   ENT_CIRCULAR        CX(n-1,0), then linear: x = C(y ^ (y << 1)), C: bit 0 ^= bit n-1
//   ENT_FULL            CX(i,j) for all i < j, lexicographic: y = x ^ (x << 1), x = prefix XOR of y
//   ENT_REVERSE_LINEAR  CX(n-2,n-1) down to CX(0,1): the same map as full
//   ENT_PAIRWISE        CX(i,i+1) for even i, then odd i: A = O E, x = E(O(y)) with
//                       E: odd bits ^= the bit below, O: even bits >= 2 ^= the bit below
//   ENT_SCA             layer r, offset o = r - 1: the circular list rotated right by
//                       o mod n, control and target swapped for odd o; in the frame
//                       z_k = y_{s+k mod n}, s = n-1-o mod n, it is a ring of CX(k, k+1)
//                       closed by CX(n-1, 0) (even o), or of CX(k+1, k) closed by
//                       CX(0, n-1) (odd o)
enum Entangler : int {
  ENT_LINEAR = 0,
  ENT_CIRCULAR = 1,
  ENT_FULL = 2,
  ENT_REVERSE_LINEAR = 3,
  ENT_PAIRWISE = 4,
  ENT_SCA = 5,
};

// The closed form of one layer's A^-1.
enum EntForm : int {
  EF_DIFF = 0,       // x = y ^ (y << 1)
  EF_WRAP_DIFF = 1,  // EF_DIFF, then bit 0 ^= bit n-1
  EF_PREFIX = 2,     // x_j = y_0 ^ ... ^ y_j
  EF_PAIRS = 3,      // z = y ^ ((y << 1) & m1), x = z ^ ((z << 1) & m2)
  EF_RING = 4,       // frame z = rot_s(y): z_0 ^= z_{n-1}, then EF_DIFF, rotated back
  EF_RING_REV = 5,   // frame z = rot_s(y): z_{n-1} ^= z_0, then suffix XOR, rotated back
};

struct EntMap {
  int form;
  int s;            // EF_RING*: the frame's origin qubit
  uint32_t m1, m2;  // EF_PAIRS: target masks of the odd-start and even-start halves
  int sh;           // index bits below the qubits (1 on the complex path: the re/im channel)
};

// x = y rotated so that bit s lands on bit 0, within n bits (0 <= s < n)
__host__ __device__ inline uint32_t rot_down(uint32_t y, int s, int n, uint32_t nmask) {
  return (uint32_t)((((uint64_t)y << (n - s)) | ((uint64_t)y >> s)) & nmask);
}
__host__ __device__ inline uint32_t rot_up(uint32_t y, int s, int n, uint32_t nmask) {
  return (uint32_t)((((uint64_t)y << s) | ((uint64_t)y >> (n - s))) & nmask);
}

// One closed form, chosen at compile time (kernels hoist the choice out of loops).
template <int F>
__host__ __device__ inline uint32_t ent_inv_f(uint32_t y, uint32_t nmask, const EntMap &e, int n) {
  if constexpr (F == EF_PREFIX) {
    uint32_t x = y;
    x ^= x << 1;
    x ^= x << 2;
    x ^= x << 4;
    x ^= x << 8;
    x ^= x << 16;
    return x & nmask;
  } else if constexpr (F == EF_WRAP_DIFF) {
    const uint32_t z = (y ^ (y << 1)) & nmask;
    return z ^ ((z >> (n - 1)) & 1u);
  } else if constexpr (F == EF_PAIRS) {
    const uint32_t z = y ^ ((y << 1) & e.m1);
    return z ^ ((z << 1) & e.m2);
  } else if constexpr (F == EF_RING) {
    uint32_t z = rot_down(y, e.s, n, nmask);
    z ^= (z >> (n - 1)) & 1u;
    return rot_up((z ^ (z << 1)) & nmask, e.s, n, nmask);
  } else if constexpr (F == EF_RING_REV) {
    uint32_t z = rot_down(y, e.s, n, nmask);
    z ^= (z & 1u) << (n - 1);
    z ^= z >> 1;
    z ^= z >> 2;
    z ^= z >> 4;
    z ^= z >> 8;
    z ^= z >> 16;
    return rot_up(z, e.s, n, nmask);
  } else {
    return (y ^ (y << 1)) & nmask;
  }
}

__host__ __device__ inline uint32_t ent_inv_q(uint32_t y, uint32_t nmask, const EntMap &e, int n) {
  switch (e.form) {
    case EF_WRAP_DIFF: return ent_inv_f<EF_WRAP_DIFF>(y, nmask, e, n);
    case EF_PREFIX: return ent_inv_f<EF_PREFIX>(y, nmask, e, n);
    case EF_PAIRS: return ent_inv_f<EF_PAIRS>(y, nmask, e, n);
    case EF_RING: return ent_inv_f<EF_RING>(y, nmask, e, n);
    case EF_RING_REV: return ent_inv_f<EF_RING_REV>(y, nmask, e, n);
    default: return ent_inv_f<EF_DIFF>(y, nmask, e, n);
  }
}

// x = A^-1 y on the qubit bits of an index with e.sh channel bits below them
// (n counts all index bits, nmask = 2^n - 1).
__host__ __device__ inline uint32_t ent_inv(uint32_t y, uint32_t nmask, const EntMap &e, int n) {
  if (e.sh == 0) return ent_inv_q(y, nmask, e, n);
  const uint32_t low = (1u << e.sh) - 1u;
  return (ent_inv_q(y >> e.sh, nmask >> e.sh, e, n - e.sh) << e.sh) | (y & low);
}

// Global bit of tile bit t under the (possibly split) strided layout; the
// FULL layout is c = tb.
__host__ __device__ inline int tile_gbit(int t, int c, int a, int k1, int gap) {
  return t < c ? t : (t - c < k1 ? a + t - c : a + gap + t - c);
}

enum StoreMode : int {
  ST_PLAIN = 0,    // out[y] = v
  ST_SCATTER = 1,  // out[A^-1 y] = v: the inverse CX chain (adjoint of LD_GATHER)
  ST_NONE = 2,
};

enum PassFlags : int {
  F_ENERGY = 1,        // accumulate an energy partial per tile
  F_LAMBDA_INIT = 2,   // lambda = table * psi (diagonal H) instead of reading lambda
  // (4 unused: tile pairing is PassArgs::pair_mask)
  F_WRITE_LAMBDA = 8,  // K_LAMBDA_XY: write lambda
  F_ACCUM = 16,        // K_LAMBDA_XY: add onto lambda already written (group chunks)
  F_COMPLEX = 64,      // the complex path (full EfficientSU2 layers: RY then RZ)
  F_MPS_SITES = 128,   // K_MPS_TAB: also write the site matrices and their derivatives
  F_MPS_TC = 256,      // K_MPS / K_MPS_GRAD at bond 16: the chunk contractions on the tensor cores
};

struct PassArgs {
  int kind, load_mode, store_mode, flags;
  int n, tb, c, a;          // register size, tile bits and bit layout (see above)
  int k1, gap;              // split layout: first-run length and the global bits skipped (0, 0: one run)
  uint32_t gate_mask;       // tile bits that carry a gate in this pass
  int layer;                // r: the RY parameter of tile bit i is p = r*pstride + qubit(i) - qoff
  int pstride;              // parameters per rotation layer (n, or 2n with RZ)
  int qoff;                 // index bits below qubit 0 (0, or 1 on the complex path)
  int zoff;                 // RZ parameter of qubit q: r*pstride + zoff + q (complex path)
  int P;                    // parameters per job
  long long tiles;          // tiles per job (a power of two)
  const void *in;           // psi input (per-job stride in_stride elements)
  long long in_stride;
  const void *lam_in;       // lambda input
  long long lam_stride;
  void *out;                // psi or lambda output
  long long out_stride;
  const void *table;        // diagonal table E(x) in amplitude precision
  long long table_stride;   // elements between the tables of consecutive jobs (0: one table for all)
  const void *cs;           // (cos(theta/2), sin(theta/2)) per job and parameter
  int job0;                 // global index of job 0 of this launch (cs, minlayer)
  EntMap em;                // this layer's entangler, x = A^-1 y (LD_GATHER, LD_L0_GATHER, ST_SCATTER)
  uint32_t pair_mask;       // launch tiles t and t ^ pair_mask next to each other (0: in order)
  int l0_kbit;              // LD_L0_GATHER: the x bit that tells the two values of x's bits above tb
  uint32_t l0_hflip;        // ... and the bits above tb that flip with it
  double *part;             // partial sums [row][tile] for this pass, per-job stride part_stride
  long long part_stride;
  double *epart;            // energy partials [tile], per-job stride part_stride
  const int *minlayer;      // per job: lowest layer with an active parameter (NULL = 0)
  // X-mask groups (K_LAMBDA_XY): group g flips mask gmask[g] and owns terms
  // [gstart[g], gstart[g+1]) with z-masks tz[] and coefficients tc[] (amplitude precision).
  const uint32_t *gmask;
  const int *gstart;
  int ngroups;
  const uint32_t *tz;
  const void *tc;
  const void *tci;  // complex path: imaginary coefficient parts (i^#Y folded in)
};

// Closed-form leading layers (gvqe_mps.cu).  After r layers the state is a
// product of D x D site matrices, D = 2^r, evaluated per amplitude from four
// tables of contracted site ranges: qubits [0, 7) (a row vector per pattern,
// stored transposed [D][128]), [7, 13) (a matrix per pattern, [64][D][D]),
// [13, 13 + h1) ([2^h1][D][D]) and [13 + h1, n) (a column vector, [2^h2][D]),
// h1 = min(9, n - 13).  Offsets in floats inside one job's table region.
constexpr int MPS_MAX_LAYERS = 4;   // bond dimension up to 16
constexpr int MPS_AUTO_LAYERS = 4;  // the default
constexpr int MPS_MIN_QUBITS = 14;
constexpr int MPS_CHUNK_BITS = 13;
// With gradients (K_MPS_TAB flag F_MPS_SITES) the region also holds the site
// matrices themselves, [q][y][a][b], and their derivatives by each layer's
// angle, [k][q][y][a][b] for k = 0..r (FP32, rounded from FP64).
struct MpsDims {
  int D, h1, h2;
  long long lo, mid, m1, r2, total;
  long long sites, dsites, total_grad;
};
__host__ __device__ inline MpsDims mps_dims(int n, int r) {
  MpsDims d;
  d.D = 1 << r;
  d.h1 = (n - MPS_CHUNK_BITS) < 9 ? (n - MPS_CHUNK_BITS) : 9;
  d.h2 = n - MPS_CHUNK_BITS - d.h1;
  const long long D = d.D;
  d.lo = 0;
  d.mid = d.lo + 128 * D;
  d.m1 = d.mid + 64 * D * D;
  d.r2 = d.m1 + (1LL << d.h1) * D * D;
  d.total = d.r2 + (1LL << d.h2) * D;
  d.sites = (d.total + 3) / 4 * 4;
  d.dsites = d.sites + (long long)n * 2 * D * D;
  d.total_grad = d.dsites + (long long)(r + 1) * n * 2 * D * D;
  return d;
}
// Gradient scratch of one job (doubles), for layer r's stage at n qubits:
// per-CTA partials of the pass over lambda (mu: [128][D], P: [64][D][D]), the
// left-contracted vector of every chunk (floats), per-block partials of the
// high qubits, their fixed-order sums, and the final gradients [k][q].
constexpr int MPS_GRAD_CTAS = 256;     // CTAs of the pass over lambda (two per SM fit at D <= 8)
constexpr int MPS_GRAD_CTAS_16 = 152;  // at D = 16 one CTA per SM fits: one wave on 152 SMs
struct MpsGradRegions {
  long long gc, nb3, v1, k;
  long long part1, lall, part3, red, fin, total;
};
__host__ __device__ inline MpsGradRegions mps_grad_regions(int n, int r) {
  MpsGradRegions g;
  const long long D = 1LL << r, chunks = 1LL << (n - MPS_CHUNK_BITS);
  const long long cap = (r >= 4) ? MPS_GRAD_CTAS_16 : MPS_GRAD_CTAS;
  g.gc = chunks < cap ? chunks : cap;
  g.nb3 = (chunks + 255) / 256;
  g.v1 = 128 * D + 64 * D * D;
  g.k = n - MPS_CHUNK_BITS;
  g.part1 = 0;
  g.lall = g.part1 + g.gc * g.v1;
  g.part3 = g.lall + (chunks * D + 1) / 2;
  g.red = g.part3 + g.k * (r + 1) * g.nb3;
  g.fin = g.red + g.v1 + g.k * (r + 1);
  g.total = g.fin + (long long)n * (r + 1);
  return g;
}

// One output of the final reduction: the sum of `count` partials starting at
// `off` inside a job's partial buffer becomes E (param < 0) or grad[param].
struct RedEntry {
  long long off;
  int count;
  int param;
};

// Shared-memory layout of one chunk of X-mask groups: [gmask][gstart][tz][tc]
// [run starts][per-term slot masks][two partner tiles of 2^tb amplitudes],
// 16-byte aligned parts (tb = 0: the group tables alone).
struct XyLayout {
  size_t gm, gs, tz, tc, runs, km, buf, total;
};
__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline XyLayout xy_layout(int ngroups, int nterm, int elem, int tb = 0) {
  XyLayout l;
  l.gm = 0;
  l.gs = align16((size_t)ngroups * 4);
  l.tz = align16(l.gs + (size_t)(ngroups + 1) * 4);
  l.tc = align16(l.tz + (size_t)nterm * 4);
  l.runs = align16(l.tc + (size_t)nterm * elem);
  l.km = align16(l.runs + (size_t)(ngroups + 1) * 4);
  l.buf = align16(l.km + (size_t)nterm * 4);
  l.total = l.buf + (tb > 0 ? ((size_t)2 * elem << tb) : 0);
  return l;
}

// Host-side launchers (gvqe_kernels.cu).  prec: 0 = float, 1 = double.
// nterm: number of terms of the X-mask group chunk (K_LAMBDA_XY only).
cudaError_t launch_pass(int prec, const PassArgs &A, int jobs, int nterm, cudaStream_t s);
// shared memory of one complex-path X/Y chunk (gvqe_kernels.cu); 1024 amplitudes per CTA
size_t xyc_smem_bytes(int prec, int ngroups, int nterm);
constexpr int XYC_AMPS_PER_CTA = 1024;
// Shared memory of the group tables of one K_LAMBDA_XY launch (the two partner
// tiles come on top: at most ~200 KiB in all is accepted).
size_t xy_smem_bytes(int prec, int ngroups, int nterm);
cudaError_t launch_trig(int prec, const double *params, long long count, void *cs, cudaStream_t s);
// K_MPS_TAB / K_MPS launches (gvqe_mps.cu, FP32 only).  K_MPS_TAB: layer = r,
// gate_mask = the qubits layer r has rotated at this stage, em = the entangler
// (EF_DIFF or EF_PREFIX), out = table region (out_stride floats per job).
// K_MPS: in = that region (in_stride), out = the state, tiles = 2^(n - 13) chunks.
// Gradient steps (layer = r, tiles = chunks; regions of mps_grad_regions inside
// the partial buffer, part_stride doubles per job):
//   K_MPS_GRAD:  in = tables, lam_in = lambda_r (lam_stride), part = per-CTA partials,
//                out = chunk vectors (floats, out_stride floats per job)
//   K_MPS_GHIGH: in = tables, lam_in = chunk vectors (lam_stride floats), part = block partials
//   K_MPS_GRED:  part = per-CTA partials, lam_in = block partials (lam_stride doubles),
//                epart = sums
//   K_MPS_GENV:  in = tables, epart = sums, out = gradients [k][q] (out_stride doubles)
cudaError_t launch_mps(int prec, const PassArgs &A, int jobs, cudaStream_t s);
cudaError_t launch_minlayer(const uint8_t *mask, int jobs, int n, int P, int none_value, int *out,
                            cudaStream_t s);
cudaError_t launch_reduce(const double *part, long long part_stride, const RedEntry *dir, int ndir,
                          const uint8_t *mask, int P, double *E, double *grad, int jobs,
                          cudaStream_t s);
cudaError_t launch_scatter_coeffs(const uint32_t *z, const double *c, int count, double *table,
                                  cudaStream_t s);
cudaError_t launch_convert_table(const double *src, float *dst, long long count, cudaStream_t s);
cudaError_t launch_expand_table(const double *src, void *dst, long long count, int prec, cudaStream_t s);
cudaError_t launch_shift_params(const double *params, int P, int jobs, const int *active,
                                int n_active, double *out, cudaStream_t s);
cudaError_t launch_shift_combine(const double *Es, int P, int jobs, const int *active, int n_active,
                                 double *E, double *grad, cudaStream_t s);
// Readout of a prepared state (gvqe_readout.cu).  Chunks of 2^readout_chunk_bits(n)
// amplitudes; RO_BINS histogram bins per CVaR search pass.
constexpr int RO_BINS = 2048;
int readout_chunk_bits(int n);
int readout_tail_parts();
// csum/cmax/cidx: [chunks], cdf: [chunks + 1]; writes stats[0] (largest p),
// stats[2] (total) and argmax[0].
cudaError_t launch_ro_modulus(int prec, const void *psi, int n, void *out, cudaStream_t s);
cudaError_t launch_ro_prob(int prec, const void *psi, int n, double *csum, double *cmax, long long *cidx,
                           double *cdf, double *stats, long long *argmax, cudaStream_t s);
cudaError_t launch_ro_sample(int prec, const void *psi, int n, const double *cdf, const double *u, int nshots,
                             long long *shots, cudaStream_t s);
// ext[1] / ext[2]: order-preserving keys of the smallest / largest E (atomic min / max).
cudaError_t launch_ro_minmax(const double *E, int n, unsigned long long *ext, cudaStream_t s);
// edges: RO_BINS + 1 device keys, the order-preserving unsigned images of
// non-decreasing bin-edge energies; gmass: RO_BINS counters; ext[1..2] as
// described in the kernel.
// below != 0: also the integer mass under the range into ext[0].
cudaError_t launch_ro_hist(int prec, const void *psi, const double *E, int n, const unsigned long long *edges,
                           unsigned long long *gmass, unsigned long long *ext, int below, cudaStream_t s);
// out[k] = E[shots[k]] for k < nshots.
cudaError_t launch_ro_gather(const double *E, const long long *shots, int nshots, double *out, cudaStream_t s);
// part: 3 * readout_tail_parts() doubles; writes stats[1].
cudaError_t launch_ro_cvar(int prec, const void *psi, const double *E, int n, double alpha, double tau,
                           double *part, double *stats, cudaStream_t s);
// Largest tile size (log2 amplitudes) whose backward pass fits in shared memory.
int max_tile_bits(int prec);
// Multiprocessors of the current device (queried once).
int num_sms_cached();
// Layer-0 gradient pass (gvqe_grad_l0.cu).  Its PassArgs use c = mb, the
// number of 1024-amplitude chunks (log2) one warp folds into a group, and
// tiles = the warps per job, which is also the number of partials per qubit.
void grad_l0_layout(int n, int prec, int *mb, long long *slots);
cudaError_t launch_grad_l0(int prec, const PassArgs &A, int jobs, cudaStream_t s);
// Dynamic shared memory (bytes) needed by one pass launch.
size_t pass_smem_bytes(int prec, int kind, int tb);

}  // namespace gvqe
