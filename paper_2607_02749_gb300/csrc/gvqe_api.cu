// gvqe_api.cu -- C ABI, Hamiltonian parsing, pass planner, workspaces and
// launch sequences of the Graph-VQE energy / gradient engine.
//
// The paths implemented here:
//   energy      forward passes of every RY layer (Section IV-B) with the
//               energy of Eq. 4 fused into the last pass (diagonal H) or a
//               separate lambda = H psi pass (X/Y strings, Eq. 6).
//   adjoint     forward passes keep every pass output; the backward walks the
//               passes in reverse, forming dE/dtheta = Im<lambda|Y_q|psi> and
//               applying RY(-theta) to lambda only (psi comes from the stored
//               outputs), then the layer-0 gradients against the analytic
//               product state.
//   param shift Eq. 13: 2 P_active + 1 energies of shifted parameter sets.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gvqe.h"
#include "gvqe_engine.cuh"
#include "gvqe_internal.h"

namespace gvqe {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define GV_CUDA(expr)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess) return fail(GVQE_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

#define GV_TRY(expr)             \
  do {                           \
    int rc_ = (expr);            \
    if (rc_ != GVQE_OK) return rc_; \
  } while (0)

// ------------------------------------------------------------ device memory --
// Device bytes held by all workspaces of this process, and an optional budget
// (gvqe_set_device_memory_limit) that reservations may not exceed.
static std::atomic<long long> g_mem_used{0};
static std::atomic<long long> g_mem_limit{0};

static long long budget_left() {
  const long long lim = g_mem_limit.load();
  return lim > 0 ? std::max(0LL, lim - g_mem_used.load()) : -1;
}

#ifdef GVQE_DEBUG
// Debug builds: a guard zone of kGuard bytes of kGuardByte on each side of every
// workspace (ptr points past the lower one); gvqe_debug_check verifies them.
constexpr size_t kGuard = 4096;
constexpr unsigned char kGuardByte = 0xA5;
static std::mutex g_guard_mu;
static std::map<char *, size_t> g_guarded;  // workspace pointer -> its bytes
#endif

int DevBuf::reserve(size_t need) {
  if (need <= bytes) return GVQE_OK;
  release();
  const long long left = budget_left();
  if (left >= 0 && (long long)need > left)
    return fail(GVQE_ENOMEM, "device workspace of %.3f GiB exceeds the %.3f GiB left of the memory limit",
                need / 1073741824.0, left / 1073741824.0);
  size_t freeb = 0, total = 0;
  GV_CUDA(cudaMemGetInfo(&freeb, &total));
  if (need > freeb)
    return fail(GVQE_ENOMEM, "device workspace of %.3f GiB does not fit in %.3f GiB free", need / 1073741824.0,
                freeb / 1073741824.0);
#ifdef GVQE_DEBUG
  void *base = nullptr;
  cudaError_t e = cudaMalloc(&base, need + 2 * kGuard);
  if (e != cudaSuccess) {
    ptr = nullptr;
    cudaGetLastError();
    return fail(GVQE_ENOMEM, "cudaMalloc(%zu): %s", need + 2 * kGuard, cudaGetErrorString(e));
  }
  e = cudaMemset(base, kGuardByte, kGuard);
  if (e == cudaSuccess) e = cudaMemset((char *)base + kGuard + need, kGuardByte, kGuard);
  if (e != cudaSuccess) {
    cudaFree(base);
    ptr = nullptr;
    return fail(GVQE_ECUDA, "guard fill: %s", cudaGetErrorString(e));
  }
  ptr = (char *)base + kGuard;
  {
    std::lock_guard<std::mutex> lk(g_guard_mu);
    g_guarded[(char *)ptr] = need;
  }
#else
  cudaError_t e = cudaMalloc(&ptr, need);
  if (e != cudaSuccess) {
    ptr = nullptr;
    cudaGetLastError();
    return fail(GVQE_ENOMEM, "cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
  }
#endif
  bytes = need;
  g_mem_used += (long long)need;
  return GVQE_OK;
}

void DevBuf::release() {
  if (ptr) {
#ifdef GVQE_DEBUG
    {
      std::lock_guard<std::mutex> lk(g_guard_mu);
      g_guarded.erase((char *)ptr);
    }
    cudaFree((char *)ptr - kGuard);
#else
    cudaFree(ptr);
#endif
    g_mem_used -= (long long)bytes;
  }
  ptr = nullptr;
  bytes = 0;
}

// ------------------------------------------------- launch accounting --
static std::atomic<long long> g_launches{0};

struct ProfRec {
  cudaEvent_t a, b;
  int kind;
  int kernels;  // kernels the step launched
  double bytes;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<ProfRec> g_prof_pending;
constexpr int PROF_KINDS = 11;  // PassKind values
static long long g_prof_n[PROF_KINDS] = {};
static double g_prof_ms[PROF_KINDS] = {};
static double g_prof_bytes[PROF_KINDS] = {};

void count_launches(int k) { g_launches += k; }

// Bytes a pass must move at minimum: every element it reads or writes, once.
static double pass_bytes(int prec, const PassArgs &A, int jobs) {
  const double S = std::ldexp(1.0, A.n) * (prec ? 8 : 4) * jobs;
  double b = 0;
  switch (A.kind) {
    case K_FWD:
    case K_WHT:
      if (A.load_mode == LD_PLAIN || A.load_mode == LD_GATHER) b += S;
      if (A.store_mode != ST_NONE) b += S;
      if (A.flags & F_ENERGY) b += S;
      break;
    case K_BWD:
      b = (A.store_mode == ST_NONE) ? 2 * S : 3 * S;
      break;
    case K_GRAD_L0:
      b = S;
      break;
    case K_LAMBDA_XY:
      b = 2 * S + ((A.flags & F_WRITE_LAMBDA) ? S : 0);
      break;
    case K_MPS:
      b = S;  // write-only
      break;
    case K_MPS_TAB:
      b = (double)mps_dims(A.n, A.layer).total * 4 * jobs;
      break;
    case K_MPS_GRAD:
      b = S;  // read lambda once
      break;
  }
  return b;
}

cudaError_t launch_step(int prec, const PassArgs &A, int jobs, int nterm, cudaStream_t s) {
  ProfRec rec{};
  bool prof;
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof = g_prof_on;
  }
  if (prof) {
    cudaEventCreate(&rec.a);
    cudaEventCreate(&rec.b);
    cudaEventRecord(rec.a, s);
  }
  const cudaError_t e = launch_pass(prec, A, jobs, nterm, s);
  const int nk = A.kind >= K_MPS ? mps_step_kernels(A) : 1;
  g_launches += nk;
  if (prof) {
    cudaEventRecord(rec.b, s);
    rec.kind = A.kind;
    rec.kernels = nk;
    rec.bytes = pass_bytes(prec, A, jobs);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_pending.push_back(rec);
  }
  return e;
}

static void prof_drain() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (ProfRec &r : g_prof_pending) {
    float ms = 0.f;
    cudaEventSynchronize(r.b);
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess && r.kind >= 0 && r.kind < PROF_KINDS) {
      g_prof_n[r.kind] += r.kernels;
      g_prof_ms[r.kind] += ms;
      g_prof_bytes[r.kind] += r.bytes;
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_prof_pending.clear();
}

// ---------------------------------------------------------------- planner --
// 2^13 FP32 / 2^12 FP64 amplitudes per tile: a backward tile (psi + lambda) is
// 64 KiB, so three CTAs share an SM, and n = 30 still takes three passes per layer.
int auto_tile_bits(int prec) { return prec ? 12 : 13; }

std::vector<LayerPass> layer_passes(int n, int prec, int tile_bits, int split) {
  std::vector<LayerPass> out;
  const int tbmax = tile_bits > 0 ? tile_bits : auto_tile_bits(prec);
  if (n <= tbmax) {
    out.push_back({n, n, n, (uint32_t)((1ull << n) - 1)});
    return out;
  }
  const int tb = tbmax;
  out.push_back({tb, tb, tb, (uint32_t)((1ull << tb) - 1)});
  // Contiguous runs of 128 bytes (carry 5 FP32 / 4 FP64); drop to 64-byte runs
  // when that saves a whole pass over the state.
  const int min_carry = prec ? 4 : 5;
  int gmax = tb - min_carry;
  const int rest = n - tb;
  int chunks = (rest + gmax - 1) / gmax;
  if ((rest + gmax) / (gmax + 1) < chunks) {
    gmax += 1;
    chunks = (rest + gmax - 1) / gmax;
  }
  int a = tb;
  for (int i = 0; i < chunks; ++i) {
    const int g = rest / chunks + (i < rest % chunks ? 1 : 0);
    const int c = tb - g;
    out.push_back({c, a, tb, (uint32_t)(((1ull << g) - 1) << c)});
    a += g;
  }
  // Two strided passes over [tb, n): the first takes [tb, tb + gA), the second
  // the top bits.  A tile of the top pass touches one 2 MiB page per combination
  // of its gate bits at or above index bit pb (stride >= 2 MiB).  Measured on
  // GB300: with 64-byte runs, a top pass over 2^9 such pages ran 1.8x slower than
  // a pass over the middle qubits, while 2^8 pages at the top ran at full speed.
  // The split layout gives the first pass [tb, tb + x) and [n - y, n) and the
  // second pass [tb + x, n - y).  Auto, when the top pass would span more than
  // 2^8 pages: the fewest top qubits y that bring the second pass down to 2^8
  // (at n = 30 RY+RZ, y = 4 and 5 measured best, 6 and 3 about 4% slower).
  // Split modes above SPLIT_ALWAYS name y itself: split = SPLIT_ALWAYS + y.
  if (chunks == 2 && split != SPLIT_NEVER) {
    LayerPass &pa = out[1], &pb_ = out[2];
    const int gA = tb - pa.c;
    const int pb = prec ? 18 : 19;
    auto pages = [&](int lo, int hi) { return std::max(0, hi - std::max(lo, pb)); };
    const int top = pages(tb + gA, n);
    int best_y = 0;
    if (split > SPLIT_ALWAYS) {
      best_y = std::min(split - SPLIT_ALWAYS, gA - 1);
    } else if (top > 8) {
      for (int y = 1; y < gA && best_y == 0; ++y)
        if (pages(tb + gA - y, n - y) <= 8) best_y = y;
    }
    if (best_y == 0 && split == SPLIT_ALWAYS && gA >= 2) best_y = gA / 2;
    if (best_y > 0) {
      const int x = gA - best_y;
      pa.k1 = x;
      pa.gap = (n - best_y) - (tb + x);
      pb_.a = tb + x;
    }
  }
  return out;
}

static int qubit_of(const LayerPass &lp, int i) { return tile_gbit(i, lp.c, lp.a, lp.k1, lp.gap); }

void set_pass_layout(PassArgs &A, const LayerPass &lp) {
  A.tb = lp.tb;
  A.c = lp.c;
  A.a = lp.a;
  A.k1 = lp.k1;
  A.gap = lp.gap;
}

// ------------------------------------------------------------- entanglers --
// The closed form of A^-1 for the entangler of layer r (1 .. reps).
EntMap ent_map(int ent, int n, int r) {
  EntMap e;
  memset(&e, 0, sizeof(e));
  e.form = EF_DIFF;
  if (n < 2) return e;  // no CNOT: the identity, which EF_DIFF is on one bit
  const uint32_t nmask = (uint32_t)((1ull << n) - 1);
  switch (ent) {
    case ENT_CIRCULAR:
      e.form = EF_WRAP_DIFF;
      break;
    case ENT_FULL:
    case ENT_REVERSE_LINEAR:
      e.form = EF_PREFIX;
      break;
    case ENT_PAIRWISE:
      e.form = EF_PAIRS;
      e.m1 = 0x55555554u & nmask;  // odd-start half: targets the even bits >= 2
      e.m2 = 0xAAAAAAAAu & nmask;  // even-start half: targets the odd bits
      break;
    case ENT_SCA: {
      const int o = (r - 1) % n;
      e.s = (n - 1 - o) % n;
      if ((r - 1) & 1)
        e.form = EF_RING_REV;
      else
        e.form = (o == 0) ? EF_WRAP_DIFF : EF_RING;  // offset 0 is the circular entangler
      break;
    }
    default:
      break;
  }
  return e;
}

// y = A x from the columns of A^-1 (Gauss-Jordan over GF(2); n <= 32).
static uint32_t ent_forward(const EntMap &e, int n, uint32_t x) {
  const uint32_t nmask = (n >= 32) ? 0xffffffffu : ((1u << n) - 1);
  // rows[j]: bit i set when bit j of A^-1 e_i is set; aug[j]: the identity
  uint32_t rows[32], aug[32];
  for (int j = 0; j < n; ++j) {
    rows[j] = 0;
    aug[j] = 1u << j;
  }
  for (int i = 0; i < n; ++i) {
    const uint32_t c = ent_inv(1u << i, nmask, e, n);
    for (int j = 0; j < n; ++j)
      if ((c >> j) & 1u) rows[j] |= 1u << i;
  }
  for (int col = 0; col < n; ++col) {
    int piv = -1;
    for (int j = col; j < n; ++j)
      if ((rows[j] >> col) & 1u) {
        piv = j;
        break;
      }
    if (piv < 0) return 0;  // not invertible: cannot happen for a CNOT product
    std::swap(rows[col], rows[piv]);
    std::swap(aug[col], aug[piv]);
    for (int j = 0; j < n; ++j)
      if (j != col && ((rows[j] >> col) & 1u)) {
        rows[j] ^= rows[col];
        aug[j] ^= aug[col];
      }
  }
  // rows is now the identity, aug = (A^-1)^-1 = A as rows: bit j of A x = parity(aug[j] & x)
  uint32_t y = 0;
  for (int j = 0; j < n; ++j) y |= (uint32_t)(__builtin_parity(aug[j] & x)) << j;
  return y;
}

// Tile pairing of a gathering pass whose tiles are y bits [0, tb): over one tile
// the x bits >= tb of x = A^-1 y flip along one vector k (or stay); the tile
// t ^ (A(k << tb) >> tb) then reads the other halves of the same sectors.
static uint32_t ent_pair_mask(const EntMap &e, int n, int tb) {
  if (n <= tb) return 0;
  const uint32_t nmask = (n >= 32) ? 0xffffffffu : ((1u << n) - 1);
  uint32_t k = 0;
  for (int i = 0; i < tb; ++i) {
    const uint32_t v = ent_inv(1u << i, nmask, e, n) >> tb;
    if (v == 0) continue;
    if (k != 0 && v != k) return 0;  // more than one direction: keep the plain order
    k = v;
  }
  if (k == 0) return 0;
  const uint32_t pm = (ent_forward(e, n, k << tb) >> tb) & (uint32_t)((1ull << (n - tb)) - 1);
  return pm == 1 ? 0 : pm;  // t ^ 1 is already the launch neighbour of t
}

// Layer-0 product-state tables of a gathering pass: x bits above tb must take
// two values across a tile, told apart by one x bit kbit <= tb.
bool ent_l0_split(const EntMap &e, int n, int tb, int *kbit, uint32_t *hflip) {
  *kbit = tb;
  *hflip = 0;
  if (n <= tb + 1) return true;
  const uint32_t nmask = (n >= 32) ? 0xffffffffu : ((1u << n) - 1);
  const uint32_t him = nmask & ~((2u << tb) - 1u);
  uint32_t h = 0, g = 0, col[32];
  for (int i = 0; i < tb; ++i) {
    col[i] = ent_inv(1u << i, nmask, e, n);
    const uint32_t v = col[i] & him;
    if (v == 0) continue;
    if (h != 0 && v != h) return false;
    h = v;
    g |= 1u << i;
  }
  if (h == 0) return true;
  for (int b = tb; b >= 0; --b) {
    bool ok = true;
    for (int i = 0; i < tb && ok; ++i) ok = (((col[i] >> b) & 1u) == ((g >> i) & 1u));
    if (ok) {
      *kbit = b;
      *hflip = h;
      return true;
    }
  }
  return false;
}

static long long tiles_of(int n, int tb) { return 1LL << (n - tb); }

// The complex path (full EfficientSU2 layers, RY then RZ on every qubit): the
// state is 2^(n+1) reals with the re/im channel as index bit 0, so the passes
// run over nb = n + 1 index bits with no gate on bit 0.  Layer 0 starts from
// |0...0> as ordinary passes (no analytic product state), every layer's passes
// store their outputs for the backward sweep, and each backward pass writes
// RY partial rows [0, tb) and RZ rows [tb, 2 tb).  Diagonal H only.
static Plan build_plan_su2(int n, int reps, int prec, int tile_bits, bool want_grad, bool diag, int ent,
                           bool state_only, int split) {
  if (state_only) want_grad = false;
  if (state_only) diag = true;
  Plan pl;
  const int nb = n + 1;
  pl.n = nb;
  pl.reps = reps;
  pl.prec = prec;
  pl.P = 2 * n * (reps + 1);
  pl.lp = layer_passes(nb, prec, tile_bits, split);
  for (LayerPass &lp : pl.lp) lp.gmask &= ~1u;  // index bit 0 is the channel
  const int p = (int)pl.lp.size();
  const long long S = 1LL << nb;
  pl.state_elems = S;
  long long poff = 0;
  auto base_args = [&](int kind, const LayerPass &lp, int r) {
    PassArgs A;
    memset(&A, 0, sizeof(A));
    A.kind = kind;
    A.n = nb;
    A.P = pl.P;
    A.pstride = 2 * n;
    A.qoff = 1;
    A.zoff = n;
    A.flags = F_COMPLEX;
    set_pass_layout(A, lp);
    A.tiles = tiles_of(nb, lp.tb);
    A.gate_mask = lp.gmask;
    A.layer = r;
    return A;
  };
  int nbuf = 0;
  const int first_state = nbuf;
  int PP0 = -1, PP1 = -1, LAM0 = -1, LAM1 = -1;
  if (want_grad) {
    nbuf += (reps + 1) * p;
    LAM0 = nbuf++;
    LAM1 = nbuf++;
  } else {
    PP0 = nbuf++;
    PP1 = nbuf++;
  }
  pl.n_bufs = nbuf;
  pl.n_states = want_grad ? (reps + 1) * p : 0;
  // ---------------- forward
  int cur = -1;
  for (int r = 0; r <= reps; ++r) {
    for (int j = 0; j < p; ++j) {
      const LayerPass &lp = pl.lp[j];
      PassStep st;
      st.A = base_args(K_FWD, lp, r);
      if (j == 0) {
        st.A.load_mode = (r == 0) ? LD_ZERO : LD_GATHER;
        if (r > 0) {
          st.A.em = ent_map(ent, n, r);
          st.A.em.sh = 1;
          st.A.pair_mask = ent_pair_mask(st.A.em, nb, lp.tb);
        }
      } else {
        st.A.load_mode = LD_PLAIN;
      }
      st.in = (r == 0 && j == 0) ? -1 : cur;
      const int out = want_grad ? first_state + r * p + j : ((j == 0) ? (cur == PP0 ? PP1 : PP0) : cur);
      st.A.store_mode = ST_PLAIN;
      if (r == reps && j == p - 1 && !want_grad && !state_only && diag) {
        st.A.store_mode = ST_NONE;
        st.A.flags |= F_ENERGY;
        st.epart_region = poff;
        pl.dir.push_back({poff, (int)st.A.tiles, -1});
        poff += st.A.tiles;
      }
      st.out = out;
      pl.steps.push_back(st);
      cur = out;
    }
  }
  // X/Y groups: lambda = H psi (and the energy) by the complex X/Y kernel
  int lam_cur = -1;
  if (!diag) {
    PassStep st;
    st.A = base_args(K_LAMBDA_XY, pl.lp[0], reps);
    st.A.tiles = std::max<long long>(1, (1LL << n) / XYC_AMPS_PER_CTA);
    st.A.gate_mask = 0;
    st.A.load_mode = LD_PLAIN;
    st.A.flags |= F_ENERGY | (want_grad ? F_WRITE_LAMBDA : 0);
    st.in = cur;
    st.out = want_grad ? LAM0 : (cur == PP0 ? PP1 : PP0);
    st.epart_region = poff;
    st.xy = true;
    pl.dir.push_back({poff, (int)st.A.tiles, -1});
    poff += st.A.tiles;
    pl.steps.push_back(st);
    lam_cur = st.out;
  }
  if (!want_grad) {
    if (state_only) pl.final_buf = cur;
    pl.part_stride = poff;
    return pl;
  }
  // ---------------- backward (every layer, layer 0 included)
  for (int r = reps; r >= 0; --r) {
    for (int j = p - 1; j >= 0; --j) {
      const LayerPass &lp = pl.lp[j];
      PassStep st;
      st.A = base_args(K_BWD, lp, r);
      st.in = first_state + r * p + j;
      if (r == reps && j == p - 1 && diag) {
        st.A.flags |= F_LAMBDA_INIT | F_ENERGY;
        st.epart_region = poff;
        pl.dir.push_back({poff, (int)st.A.tiles, -1});
        poff += st.A.tiles;
        st.lam = -1;
      } else {
        st.lam = lam_cur;
      }
      const int out = (lam_cur == LAM0) ? LAM1 : LAM0;
      st.out = out;
      if (j == 0 && r > 0) {
        st.A.store_mode = ST_SCATTER;
        st.A.em = ent_map(ent, n, r);
        st.A.em.sh = 1;
        st.A.pair_mask = ent_pair_mask(st.A.em, nb, lp.tb);
      } else {
        st.A.store_mode = (j == 0) ? ST_NONE : ST_PLAIN;  // nothing runs before layer 0
      }
      st.part_region = poff;
      for (int i = 0; i < lp.tb; ++i) {
        if (!((lp.gmask >> i) & 1u)) continue;
        const int q = qubit_of(lp, i) - 1;
        const int py = r * 2 * n + q, pz = r * 2 * n + n + q;
        pl.param_dir[py] = {poff + (long long)i * st.A.tiles, (int)st.A.tiles, py};
        pl.param_dir[pz] = {poff + (long long)(lp.tb + i) * st.A.tiles, (int)st.A.tiles, pz};
      }
      poff += 2LL * lp.tb * st.A.tiles;
      pl.steps.push_back(st);
      lam_cur = out;
    }
  }
  pl.part_stride = poff;
  for (auto &kv : pl.param_dir) pl.dir.push_back(kv.second);
  return pl;
}

// Build the ordered pass list for one (n, reps, precision) and what is requested.
int mps_layers_for(int n, int reps, int prec, int ent, int gates, int want) {
  if (want < 0 || prec != 0 || gates != 1 || n < MPS_MIN_QUBITS || reps < 2) return 0;
  int R = std::min(want > 0 ? std::min(want, MPS_MAX_LAYERS) : MPS_AUTO_LAYERS, reps - 1);
  for (int r = 1; r <= R; ++r) {
    const EntMap e = ent_map(ent, n, r);
    if (e.sh != 0 || (e.form != EF_DIFF && e.form != EF_PREFIX)) return 0;
  }
  return R;
}

Plan build_plan(int n, int reps, int prec, int tile_bits, bool want_grad, bool diag, bool tile_grad_l0,
                bool state_only, int ent, int gates, int split, int xy_tb, int mps_layers, bool mps_tc) {
  if (gates == 2) return build_plan_su2(n, reps, prec, tile_bits, want_grad, diag, ent, state_only, split);
  Plan pl;
  pl.n = n;
  pl.reps = reps;
  pl.prec = prec;
  pl.P = n * (reps + 1);
  pl.lp = layer_passes(n, prec, tile_bits, split);
  const int p = (int)pl.lp.size();
  const int tbA = pl.lp[0].tb;
  const long long S = 1LL << n;
  pl.state_elems = S;
  long long poff = 0;  // partial offset (doubles) inside one job's partial buffer
  auto base_args = [&](int kind) {
    PassArgs A;
    memset(&A, 0, sizeof(A));
    A.kind = kind;
    A.n = n;
    A.P = pl.P;
    A.pstride = n;
    return A;
  };
  auto set_layout = [&](PassArgs &A, const LayerPass &lp) {
    set_pass_layout(A, lp);
    A.tiles = tiles_of(n, lp.tb);
  };
  // Buffer ids: stored pass outputs (gradient path) or a forward ping-pong
  // pair (energy path), the lambda ping-pong pair, and psi_0 for X/Y terms at reps = 0.
  // closed-form leading layers 1..R; with gradients, theirs come from lambda_R
  // and the matrix product (mgrad), so only layer R's final state is stored
  const int R = (mps_layers > 0 && reps >= 2) ? std::min(mps_layers, reps - 1) : 0;
  const bool mgrad = want_grad && !state_only && R >= 1 && R <= MPS_MAX_LAYERS;
  int nb = 0;
  const int first_state = nb;
  if (want_grad) nb += mgrad ? 1 + (reps - R) * p : reps * p;
  // buffer of the stored state after pass j of layer r (gradient path)
  auto state_id = [&](int r, int j) {
    if (!mgrad) return first_state + (r - 1) * p + j;
    return (r == R) ? first_state : first_state + 1 + (r - R - 1) * p + j;
  };
  int PP0 = -1, PP1 = -1;
  if (!want_grad && reps > 0) {
    PP0 = nb++;
    PP1 = nb++;
  }
  int LAM0 = -1, LAM1 = -1;
  if (state_only) {  // the forward passes alone, the final state kept in a buffer
    want_grad = false;
    diag = false;
  }
  if (want_grad || (!diag && !state_only)) LAM0 = nb++;
  if (want_grad) LAM1 = nb++;
  int XYB = -1;
  if (reps == 0 && !diag) XYB = nb++;
  pl.n_bufs = nb;
  pl.n_states = want_grad ? (mgrad ? 1 + (reps - R) * p : reps * p) : 0;

  auto add_E_region = [&](long long tiles) {
    pl.dir.push_back({poff, (int)tiles, -1});
    poff += tiles;
  };

  // ---------------- forward
  int cur = -1;  // buffer holding the current state
  int last_state = -1;
  if (reps == 0) {
    if (!diag) {
      PassStep st;
      st.A = base_args(K_FWD);
      set_layout(st.A, pl.lp[0]);
      st.A.load_mode = LD_L0;
      st.A.store_mode = ST_PLAIN;
      st.A.gate_mask = 0;
      st.A.layer = 0;
      st.out = XYB;
      pl.steps.push_back(st);
      last_state = XYB;
    } else if (!want_grad) {
      PassStep st;
      st.A = base_args(K_FWD);
      set_layout(st.A, pl.lp[0]);
      st.A.load_mode = LD_L0;
      st.A.store_mode = ST_NONE;
      st.A.flags = F_ENERGY;
      st.A.gate_mask = 0;
      st.epart_region = poff;
      add_E_region(st.A.tiles);
      pl.steps.push_back(st);
    }
  }
  // closed-form leading layers: every stored state of layers 1..R (gradient
  // path without mgrad), or layer R's final state alone (energy path; mgrad,
  // whose table region then also keeps the site matrices for the gradients)
  pl.mps_layers = R;
  pl.mps_grad = mgrad;
  pl.mps_tc = R == MPS_MAX_LAYERS && mps_tc;
  for (int r = 1; r <= R; ++r) {
    uint32_t rot = 0;
    for (int j = 0; j < p; ++j) {
      const LayerPass &lp = pl.lp[j];
      for (int i = 0; i < lp.tb; ++i)
        if ((lp.gmask >> i) & 1u) rot |= 1u << qubit_of(lp, i);
      if ((!want_grad || mgrad) && !(r == R && j == p - 1)) continue;
      const MpsDims md = mps_dims(n, r);
      pl.mps_elems = std::max(pl.mps_elems, ((mgrad ? md.total_grad : md.total) + 63) / 64 * 64);
      PassStep tab;
      tab.A = base_args(K_MPS_TAB);
      tab.A.layer = r;
      tab.A.gate_mask = rot;
      tab.A.em = ent_map(ent, n, r);
      tab.A.tiles = 1;
      if (mgrad) tab.A.flags |= F_MPS_SITES;
      pl.steps.push_back(tab);
      PassStep st = tab;
      st.A.kind = K_MPS;
      st.A.flags = (r == MPS_MAX_LAYERS && mps_tc) ? F_MPS_TC : 0;
      st.A.tiles = 1LL << (n - MPS_CHUNK_BITS);
      st.A.store_mode = ST_PLAIN;
      st.out = want_grad ? state_id(r, j) : PP0;
      pl.steps.push_back(st);
      cur = st.out;
    }
  }
  for (int r = R + 1; r <= reps; ++r) {
    for (int j = 0; j < p; ++j) {
      const LayerPass &lp = pl.lp[j];
      PassStep st;
      st.A = base_args(K_FWD);
      set_layout(st.A, lp);
      st.A.gate_mask = lp.gmask;
      st.A.layer = r;
      if (j == 0) {
        st.A.load_mode = (r == 1) ? LD_L0_GATHER : LD_GATHER;
        st.A.em = ent_map(ent, n, r);
        st.A.pair_mask = ent_pair_mask(st.A.em, n, lp.tb);
        if (r == 1) ent_l0_split(st.A.em, n, lp.tb, &st.A.l0_kbit, &st.A.l0_hflip);
      } else {
        st.A.load_mode = LD_PLAIN;
      }
      st.in = (r == 1 && j == 0) ? -1 : cur;
      int out;
      if (want_grad) {
        out = state_id(r, j);
      } else {
        // the gathering first pass writes the other buffer; later passes run in place
        out = (j == 0) ? (cur == PP0 ? PP1 : PP0) : cur;
      }
      st.A.store_mode = ST_PLAIN;
      const bool last = (r == reps && j == p - 1);
      if (last && diag && !want_grad) {
        st.A.store_mode = ST_NONE;
        st.A.flags |= F_ENERGY;
        st.epart_region = poff;
        add_E_region(st.A.tiles);
      }
      st.out = out;
      pl.steps.push_back(st);
      cur = out;
    }
  }
  if (reps > 0) last_state = cur;
  if (state_only) {
    pl.final_buf = last_state;
    pl.part_stride = 0;
    return pl;
  }

  // X/Y energy (and lambda) for a non-diagonal H
  int lam_cur = -1;
  if (!diag) {
    PassStep st;
    st.A = base_args(K_LAMBDA_XY);
    // the X-mask pass may take its own tile size (fewer qubits than n: the whole register)
    const int tbx = xy_tb > 0 ? std::min(std::min(xy_tb, max_tile_bits(prec)), n) : tbA;
    st.A.tb = tbx;
    st.A.c = tbx;
    st.A.a = tbx;
    st.A.tiles = tiles_of(n, tbx);
    st.A.load_mode = LD_PLAIN;
    st.A.flags = F_ENERGY | (want_grad ? F_WRITE_LAMBDA : 0);
    st.in = last_state;
    st.out = LAM0;
    st.epart_region = poff;
    st.xy = true;
    add_E_region(st.A.tiles);
    pl.steps.push_back(st);
    lam_cur = LAM0;
  }

  if (want_grad) {
    // ---------------- backward
    for (int r = reps; r >= (mgrad ? R + 1 : 1); --r) {
      for (int j = p - 1; j >= 0; --j) {
        const LayerPass &lp = pl.lp[j];
        PassStep st;
        st.A = base_args(K_BWD);
        set_layout(st.A, lp);
        st.A.gate_mask = lp.gmask;
        st.A.layer = r;
        st.in = state_id(r, j);
        const bool first = (r == reps && j == p - 1);
        if (first && diag) {
          st.A.flags |= F_LAMBDA_INIT | F_ENERGY;
          st.epart_region = poff;
          add_E_region(st.A.tiles);
          st.lam = -1;
        } else {
          st.lam = lam_cur;
        }
        const int out = (lam_cur == LAM0) ? LAM1 : LAM0;
        st.out = out;
        if (j == 0) {
          st.A.store_mode = ST_SCATTER;
          st.A.em = ent_map(ent, n, r);
          st.A.pair_mask = ent_pair_mask(st.A.em, n, lp.tb);
        } else {
          st.A.store_mode = ST_PLAIN;
        }
        st.part_region = poff;
        // partial rows for gate bits: [tile bit][tile]
        for (int i = 0; i < lp.tb; ++i) {
          if (!((lp.gmask >> i) & 1u)) continue;
          const int q = qubit_of(lp, i);
          pl.param_dir[r * n + q] = {poff + (long long)i * st.A.tiles, (int)st.A.tiles, r * n + q};
        }
        poff += (long long)lp.tb * st.A.tiles;
        pl.steps.push_back(st);
        lam_cur = out;
      }
    }
    if (mgrad) {
      // ---------------- gradients of layers 0..R from lambda_R (closed form)
      const MpsGradRegions g = mps_grad_regions(n, R);
      const long long base = poff;
      poff += g.total;
      for (int kind : {K_MPS_GRAD, K_MPS_GHIGH, K_MPS_GRED, K_MPS_GENV}) {
        PassStep st;
        st.A = base_args(kind);
        st.A.layer = R;
        st.A.tiles = 1LL << (n - MPS_CHUNK_BITS);
        st.A.em = ent_map(ent, n, R);
        st.lam = (kind == K_MPS_GRAD) ? lam_cur : -1;
        if (kind == K_MPS_GRAD && R == MPS_MAX_LAYERS && mps_tc) st.A.flags |= F_MPS_TC;
        st.part_region = base;
        pl.steps.push_back(st);
      }
      for (int k = 0; k <= R; ++k)
        for (int q = 0; q < n; ++q) pl.param_dir[k * n + q] = {base + g.fin + (long long)k * n + q, 1, k * n + q};
      pl.part_stride = poff;
      for (auto &kv : pl.param_dir) pl.dir.push_back(kv.second);
      return pl;
    }
    // ---------------- layer-0 gradients
    PassStep st;
    st.A = base_args(K_GRAD_L0);
    st.A.tb = tbA;
    st.A.a = tbA;
    if (n > 9 && !tile_grad_l0) {  // n <= 9 runs in the whole-register kernel
      int mb = 0;
      long long slots = 1;
      grad_l0_layout(n, prec, &mb, &slots);
      st.A.c = mb;
      st.A.tiles = slots;
    } else {
      st.A.c = tbA;
      st.A.tiles = tiles_of(n, tbA);
    }
    st.A.layer = 0;
    if (reps == 0 && diag) {
      st.A.flags = F_LAMBDA_INIT | F_ENERGY;
      st.epart_region = poff;
      add_E_region(st.A.tiles);
      st.lam = -1;
    } else {
      st.lam = lam_cur;
    }
    st.part_region = poff;
    for (int q = 0; q < n; ++q) pl.param_dir[q] = {poff + (long long)q * st.A.tiles, (int)st.A.tiles, q};
    poff += (long long)n * st.A.tiles;
    pl.steps.push_back(st);
  }
  pl.part_stride = poff;
  for (auto &kv : pl.param_dir) pl.dir.push_back(kv.second);
  return pl;
}

std::string describe_plan(const Plan &pl) {
  std::string s;
  char buf[256];
  snprintf(buf, sizeof(buf), "n=%d reps=%d prec=%s passes_per_layer=%zu steps=%zu partials_per_job=%lld\n", pl.n,
           pl.reps, pl.prec ? "fp64" : "fp32", pl.lp.size(), pl.steps.size(), pl.part_stride);
  s += buf;
  for (size_t j = 0; j < pl.lp.size(); ++j) {
    const LayerPass &lp = pl.lp[j];
    // gate bits as runs of consecutive index bits: [lo,hi] or [lo,hi]+[lo2,hi2] (split)
    std::string runs;
    int lo = -1, prev = -2;
    for (int i = 0; i <= lp.tb; ++i) {
      const int q = (i < lp.tb && ((lp.gmask >> i) & 1u)) ? qubit_of(lp, i) : -1;
      if (lo >= 0 && q != prev + 1) {
        snprintf(buf, sizeof(buf), "%s[%d,%d]", runs.empty() ? "" : "+", lo, prev);
        runs += buf;
        lo = -1;
      }
      if (q >= 0 && lo < 0) lo = q;
      prev = q;
    }
    if (runs.empty()) runs = "[-1,-1]";
    snprintf(buf, sizeof(buf), "  layer pass %zu: tile_bits=%d carry=%d high_start=%d qubits=%s split=%d,%d tiles=%lld\n",
             j, lp.tb, lp.c, lp.a, runs.c_str(), lp.k1, lp.gap, tiles_of(pl.n, lp.tb));
    s += buf;
  }
  if (pl.mps_layers > 0) {
    snprintf(buf, sizeof(buf), "  closed-form layers 1..%d (bond dimension up to %d), %lld table floats per job%s\n",
             pl.mps_layers, 1 << pl.mps_layers, pl.mps_elems,
             !pl.mps_grad ? (pl.mps_tc ? " (tensor cores, TF32 split)" : "")
             : pl.mps_tc  ? "; their gradients from lambda and the matrix product (tensor cores, TF32 split)"
                          : "; their gradients from lambda and the matrix product");
    s += buf;
  }
  static const char *kinds[] = {"fwd",     "bwd",       "grad_l0",   "lambda_xy", "wht",     "mps",
                                "mps_tab", "mps_grad", "mps_ghigh", "mps_gred", "mps_genv"};
  for (const PassStep &st : pl.steps) {
    snprintf(buf, sizeof(buf), "  %-9s layer=%d tb=%d c=%d a=%d gates=0x%x load=%d store=%d flags=0x%x in=%d lam=%d out=%d\n",
             kinds[st.A.kind], st.A.layer, st.A.tb, st.A.c, st.A.a, st.A.gate_mask, st.A.load_mode, st.A.store_mode,
             st.A.flags, st.in, st.lam, st.out);
    s += buf;
  }
  return s;
}

}  // namespace gvqe

using namespace gvqe;

// ------------------------------------------------------------ Hamiltonian --
static int parse_hamiltonian(gvqe_hamiltonian_s *h, int n, int m, const char *pauli, const double *coeffs) {
  std::map<uint32_t, double> diag;
  std::map<uint32_t, std::map<uint32_t, double>> groups;
  std::map<uint32_t, std::map<uint32_t, std::pair<double, double>>> cgroups;  // complex path
  h->n_dropped = 0;
  h->abs_sum = 0.0;
  for (int k = 0; k < m; ++k) {
    uint32_t mx = 0, mz = 0;
    int ny = 0;
    for (int q = 0; q < n; ++q) {
      const char L = pauli[(size_t)k * n + q];
      switch (L) {
        case 'I': break;
        case 'X': mx |= 1u << q; break;
        case 'Y': mx |= 1u << q; mz |= 1u << q; ++ny; break;
        case 'Z': mz |= 1u << q; break;
        default:
          return fail(GVQE_EINVAL, "term %d: letter '%c' at position %d is not one of I, X, Y, Z", k,
                      (L >= 32 && L < 127) ? L : '?', q);
      }
    }
    const double c = coeffs[k];
    if (!std::isfinite(c)) return fail(GVQE_EINVAL, "term %d: coefficient is not finite", k);
    h->abs_sum += std::fabs(c);
    if (mx != 0) {  // i^ny = 1, i, -1, -i for ny = 0, 1, 2, 3 (mod 4)
      auto &v = cgroups[mx][mz];
      const int r4 = ny % 4;
      if (r4 == 0) v.first += c;
      if (r4 == 1) v.second += c;
      if (r4 == 2) v.first -= c;
      if (r4 == 3) v.second -= c;
    }
    if (mx == 0) {
      diag[mz] += c;
    } else if (ny & 1) {
      h->n_dropped += 1;  // odd #Y: purely imaginary on real states, contributes exactly zero
    } else {
      // P|u> = i^ny (-1)^popcount(u & z') |u ^ m>, i^ny = +1 (ny = 0 mod 4) or -1 (ny = 2 mod 4)
      groups[mx][mz] += (ny % 4 == 0) ? c : -c;
    }
  }
  h->dz.clear();
  h->dc.clear();
  for (auto &kv : diag) {
    h->dz.push_back(kv.first);
    h->dc.push_back(kv.second);
  }
  h->gm.clear();
  h->gs.clear();
  h->tz.clear();
  h->tc.clear();
  h->n_grouped = 0;
  for (auto &g : groups) {
    h->gm.push_back(g.first);
    h->gs.push_back((int)h->tz.size());
    for (auto &t : g.second) {
      h->tz.push_back(t.first);
      h->tc.push_back(t.second);
      h->n_grouped += 1;
    }
  }
  h->gs.push_back((int)h->tz.size());
  h->cgm.clear();
  h->cgs.clear();
  h->ctz.clear();
  h->ctr.clear();
  h->cti.clear();
  for (auto &g : cgroups) {
    h->cgm.push_back(g.first);
    h->cgs.push_back((int)h->ctz.size());
    for (auto &t : g.second) {
      h->ctz.push_back(t.first);
      h->ctr.push_back(t.second.first);
      h->cti.push_back(t.second.second);
    }
  }
  h->cgs.push_back((int)h->ctz.size());
  return GVQE_OK;
}

// Build the FP64 diagonal table E(x) = sum_z chat[z] (-1)^popcount(x & z): scatter
// the merged coefficients, then Walsh-Hadamard passes on the device.
// An NVTX range around one public call (visible to Nsight tools; free otherwise).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

// A table built in steps: its buffer is released again unless the build
// completes, so a failed call (say, over the memory limit) leaves no half-built
// table behind for the next call to trust.
struct PendingBuf {
  DevBuf &b;
  bool done = false;
  explicit PendingBuf(DevBuf &x) : b(x) {}
  ~PendingBuf() {
    if (!done) b.release();
  }
};

static int build_table64(gvqe_hamiltonian_s *h, cudaStream_t s) {
  if (h->T64.ptr) return GVQE_OK;
  const int n = h->n;
  const size_t S = (size_t)1 << n;
  PendingBuf guard(h->T64);
  GV_TRY(h->T64.reserve(S * 8));
  GV_CUDA(cudaMemsetAsync(h->T64.ptr, 0, S * 8, s));
  if (!h->dz.empty()) {
    DevBuf tmp;
    PendingBuf tmp_guard(tmp);  // always released
    const size_t cnt = h->dz.size();
    GV_TRY(tmp.reserve(cnt * (4 + 8)));
    uint32_t *dz = (uint32_t *)tmp.ptr;
    double *dc = (double *)((char *)tmp.ptr + ((cnt * 4 + 15) / 16) * 16);
    if (((cnt * 4 + 15) / 16) * 16 + cnt * 8 > tmp.bytes) {
      tmp.release();
      GV_TRY(tmp.reserve(((cnt * 4 + 15) / 16) * 16 + cnt * 8));
      dz = (uint32_t *)tmp.ptr;
      dc = (double *)((char *)tmp.ptr + ((cnt * 4 + 15) / 16) * 16);
    }
    GV_CUDA(cudaMemcpyAsync(dz, h->dz.data(), cnt * 4, cudaMemcpyHostToDevice, s));
    GV_CUDA(cudaMemcpyAsync(dc, h->dc.data(), cnt * 8, cudaMemcpyHostToDevice, s));
    GV_CUDA(launch_scatter_coeffs(dz, dc, (int)cnt, (double *)h->T64.ptr, s));
    std::vector<LayerPass> lps = layer_passes(n, 1, 0);
    for (const LayerPass &lp : lps) {
      PassArgs A;
      memset(&A, 0, sizeof(A));
      A.kind = K_WHT;
      A.load_mode = LD_PLAIN;
      A.store_mode = ST_PLAIN;
      A.n = n;
      set_pass_layout(A, lp);
      A.tiles = 1LL << (n - lp.tb);
      A.gate_mask = lp.gmask;
      A.in = h->T64.ptr;
      A.out = h->T64.ptr;
      A.P = 1;
      GV_CUDA(launch_step(1, A, 1, 0, s));
    }
    GV_CUDA(cudaStreamSynchronize(s));
  } else {
    GV_CUDA(cudaStreamSynchronize(s));
  }
  guard.done = true;
  return GVQE_OK;
}

static int ensure_tables(gvqe_hamiltonian_s *h, int prec, cudaStream_t s, bool cplx = false) {
  GV_TRY(build_table64(h, s));
  if (cplx) {
    if (!h->TC[prec].ptr) {
      const size_t S = (size_t)1 << h->n;
      PendingBuf guard(h->TC[prec]);
      GV_TRY(h->TC[prec].reserve(S * 2 * (prec ? 8 : 4)));
      GV_CUDA(launch_expand_table((const double *)h->T64.ptr, h->TC[prec].ptr, (long long)S, prec, s));
      GV_CUDA(cudaStreamSynchronize(s));
      guard.done = true;
    }
    if (h->cgm.empty()) return GVQE_OK;
    if (!prec && !h->T32.ptr) {  // the X/Y kernel reads the plain table
      const size_t S = (size_t)1 << h->n;
      PendingBuf guard(h->T32);
      GV_TRY(h->T32.reserve(S * 4));
      GV_CUDA(launch_convert_table((const double *)h->T64.ptr, (float *)h->T32.ptr, (long long)S, s));
      GV_CUDA(cudaStreamSynchronize(s));
      guard.done = true;
    }
    if (!h->CG.ptr) {
      PendingBuf guard(h->CG);
      const size_t ng = h->cgm.size(), nt = h->ctz.size();
      auto up = [](size_t b) { return (b + 15) / 16 * 16; };
      const size_t o_gm = 0, o_gs = up(ng * 4), o_tz = o_gs + up((ng + 1) * 4);
      const size_t o_r64 = o_tz + up(nt * 4), o_i64 = o_r64 + nt * 8, o_r32 = o_i64 + nt * 8;
      const size_t o_i32 = o_r32 + up(nt * 4), total = o_i32 + up(nt * 4) + 16;
      GV_TRY(h->CG.reserve(total));
      char *b = (char *)h->CG.ptr;
      std::vector<float> r32(h->ctr.begin(), h->ctr.end()), i32(h->cti.begin(), h->cti.end());
      GV_CUDA(cudaMemcpy(b + o_gm, h->cgm.data(), ng * 4, cudaMemcpyHostToDevice));
      GV_CUDA(cudaMemcpy(b + o_gs, h->cgs.data(), (ng + 1) * 4, cudaMemcpyHostToDevice));
      GV_CUDA(cudaMemcpy(b + o_tz, h->ctz.data(), nt * 4, cudaMemcpyHostToDevice));
      GV_CUDA(cudaMemcpy(b + o_r64, h->ctr.data(), nt * 8, cudaMemcpyHostToDevice));
      GV_CUDA(cudaMemcpy(b + o_i64, h->cti.data(), nt * 8, cudaMemcpyHostToDevice));
      GV_CUDA(cudaMemcpy(b + o_r32, r32.data(), nt * 4, cudaMemcpyHostToDevice));
      GV_CUDA(cudaMemcpy(b + o_i32, i32.data(), nt * 4, cudaMemcpyHostToDevice));
      h->d_cgm = (uint32_t *)(b + o_gm);
      h->d_cgs = (int *)(b + o_gs);
      h->d_ctz = (uint32_t *)(b + o_tz);
      h->d_ctr[1] = b + o_r64;
      h->d_cti[1] = b + o_i64;
      h->d_ctr[0] = b + o_r32;
      h->d_cti[0] = b + o_i32;
      guard.done = true;
    }
    return GVQE_OK;
  }
  if (!prec && !h->T32.ptr) {
    const size_t S = (size_t)1 << h->n;
    PendingBuf guard(h->T32);
    GV_TRY(h->T32.reserve(S * 4));
    GV_CUDA(launch_convert_table((const double *)h->T64.ptr, (float *)h->T32.ptr, (long long)S, s));
    GV_CUDA(cudaStreamSynchronize(s));
    guard.done = true;
  }
  // X-mask group tables
  if (!h->gm.empty() && !h->G.ptr) {
    PendingBuf guard(h->G);
    const size_t ng = h->gm.size(), nt = h->tz.size();
    const size_t o_gm = 0, o_gs = ((ng * 4 + 15) / 16) * 16;
    const size_t o_tz = o_gs + (((ng + 1) * 4 + 15) / 16) * 16;
    const size_t o_t64 = o_tz + ((nt * 4 + 15) / 16) * 16;
    const size_t o_t32 = o_t64 + nt * 8;
    const size_t total = o_t32 + ((nt * 4 + 15) / 16) * 16 + 16;
    GV_TRY(h->G.reserve(total));
    char *b = (char *)h->G.ptr;
    std::vector<float> t32(h->tc.begin(), h->tc.end());
    GV_CUDA(cudaMemcpy(b + o_gm, h->gm.data(), ng * 4, cudaMemcpyHostToDevice));
    GV_CUDA(cudaMemcpy(b + o_gs, h->gs.data(), (ng + 1) * 4, cudaMemcpyHostToDevice));
    GV_CUDA(cudaMemcpy(b + o_tz, h->tz.data(), nt * 4, cudaMemcpyHostToDevice));
    GV_CUDA(cudaMemcpy(b + o_t64, h->tc.data(), nt * 8, cudaMemcpyHostToDevice));
    GV_CUDA(cudaMemcpy(b + o_t32, t32.data(), nt * 4, cudaMemcpyHostToDevice));
    h->d_gm = (uint32_t *)(b + o_gm);
    h->d_gs = (int *)(b + o_gs);
    h->d_tz = (uint32_t *)(b + o_tz);
    h->d_tc64 = (double *)(b + o_t64);
    h->d_tc32 = (float *)(b + o_t32);
    guard.done = true;
  }
  return GVQE_OK;
}

// --------------------------------------------------------- plan execution --
Plan *gvqe::get_plan(gvqe_ansatz_s *a, int prec, bool want_grad, bool diag, bool state_only, bool allow_mps) {
  const int key = prec | (want_grad ? 2 : 0) | (diag ? 4 : 0) | (state_only ? 8 : 0) | (a->gates == 2 ? 16 : 0) |
                  (allow_mps ? 0 : 32);
  auto it = a->plans.find(key);
  const int tb = eff_tile_bits(a, prec);
  if (it != a->plans.end() && it->second.tile_bits == tb) return &it->second;
  const int mps = allow_mps ? mps_layers_for(a->n, a->reps, prec, a->ent, a->gates, a->mps) : 0;
  Plan pl = build_plan(a->n, a->reps, prec, tb, want_grad, diag, false, state_only, a->ent, a->gates,
                       eff_split(a, prec), eff_xy_tb(a, prec), mps, a->mps_tc >= 0);
  pl.tile_bits = tb;
  a->plans[key] = std::move(pl);
  return &a->plans[key];
}

static int upload_dir(Plan *pl) {
  if (pl->d_dir.ptr && pl->d_dir_count == (int)pl->dir.size()) return GVQE_OK;
  GV_TRY(pl->d_dir.reserve(sizeof(RedEntry) * std::max<size_t>(1, pl->dir.size())));
  GV_CUDA(cudaMemcpy(pl->d_dir.ptr, pl->dir.data(), sizeof(RedEntry) * pl->dir.size(), cudaMemcpyHostToDevice));
  pl->d_dir_count = (int)pl->dir.size();
  return GVQE_OK;
}

// Run the plan for `batch` parameter vectors (already converted to cs on device).
// With a state-only plan, *state receives job 0's final state (batch must be 1).
static int run_plan(gvqe_ansatz_s *a, gvqe_hamiltonian_s *h, Plan *pl, const void *cs_all, const uint8_t *mask,
                    int batch, double *E, double *grad, const int *minlayer, cudaStream_t s,
                    void **state = nullptr) {
  const int prec = pl->prec;
  const size_t es = prec ? 8 : 4;
  const long long S = pl->state_elems;
  GV_TRY(upload_dir(pl));
  // jobs per launch: enough tiles to fill the GPU, bounded by memory
  const long long tilesA = 1LL << (pl->n - pl->lp[0].tb);
  int J = (int)std::min<long long>(batch, std::max<long long>(1, 4096 / tilesA));
  const size_t per_job = (size_t)pl->n_bufs * S * es + (size_t)pl->part_stride * 8 + (size_t)pl->mps_elems * 4;
  size_t freeb = 0, total = 0;
  GV_CUDA(cudaMemGetInfo(&freeb, &total));
  size_t have = freeb + a->ws.bytes;
  const long long left = budget_left();
  if (left >= 0) have = std::min(have, (size_t)left + a->ws.bytes + ((size_t)512 << 20));
  const size_t budget = have > (size_t)512 << 20 ? have - ((size_t)512 << 20) : 0;
  if (per_job > budget)
    return fail(GVQE_ENOMEM, "one evaluation needs %.3f GiB of workspace, %.3f GiB available", per_job / 1073741824.0,
                budget / 1073741824.0);
  J = (int)std::max<size_t>(1, std::min<size_t>((size_t)J, budget / per_job));
  const size_t need = per_job * (size_t)J + 256;
  GV_TRY(a->ws.reserve(need));
  char *base = (char *)a->ws.ptr;
  double *part = (double *)base;
  char *bufs = base + (((size_t)pl->part_stride * 8 * J + 255) / 256) * 256;
  auto buf_ptr = [&](int id) -> void * {
    if (id < 0) return nullptr;
    return bufs + (size_t)id * J * S * es;  // buffer id, job slots contiguous
  };
  // closed-form layer tables after the state buffers (a multiple of 64 floats per job)
  float *mps_tab = (float *)(bufs + (size_t)pl->n_bufs * J * S * es);
  const bool cplx = a->gates == 2;
  const void *table = h ? (cplx ? h->TC[prec].ptr : (prec ? h->T64.ptr : h->T32.ptr)) : nullptr;
  const void *tc = h ? (prec ? (const void *)h->d_tc64 : (const void *)h->d_tc32) : nullptr;
  if (state) *state = buf_ptr(pl->final_buf);
  for (int j0 = 0; j0 < batch; j0 += J) {
    const int jobs = std::min(J, batch - j0);
    for (const PassStep &st : pl->steps) {
      PassArgs A = st.A;
      A.job0 = j0;
      A.cs = cs_all;
      A.table = table;
      A.in = buf_ptr(st.in);
      A.in_stride = S;
      A.lam_in = buf_ptr(st.lam);
      A.lam_stride = S;
      A.out = buf_ptr(st.out);
      A.out_stride = S;
      A.part = part + (st.part_region >= 0 ? st.part_region : 0);
      A.epart = part + (st.epart_region >= 0 ? st.epart_region : 0);
      A.part_stride = pl->part_stride;
      A.minlayer = minlayer;
      if (A.kind == K_MPS_TAB) {
        A.out = mps_tab;
        A.out_stride = pl->mps_elems;
      } else if (A.kind >= K_MPS) {
        A.in = mps_tab;
        A.in_stride = pl->mps_elems;
        if (A.kind >= K_MPS_GRAD) {
          // the chunk vectors (floats) inside this step's partial region
          const MpsGradRegions g = mps_grad_regions(A.n, A.layer);
          float *lall = reinterpret_cast<float *>(A.part + g.lall);
          if (A.kind == K_MPS_GRAD) {
            A.out = lall;
            A.out_stride = pl->part_stride * 2;
          } else if (A.kind == K_MPS_GHIGH) {
            A.lam_in = lall;
            A.lam_stride = pl->part_stride * 2;
          }
        }
      }
      if (!st.xy) {
        GV_CUDA(launch_step(prec, A, jobs, 0, s));
        continue;
      }
      // X-mask groups in chunks that fit in shared memory; the last chunk forms the energy.
      // (the complex path uses its own groups, which keep odd-#Y strings, and the plain table)
      if (cplx) A.table = prec ? h->T64.ptr : h->T32.ptr;
      const std::vector<uint32_t> &gmv = cplx ? h->cgm : h->gm;
      const std::vector<int> &gsv = cplx ? h->cgs : h->gs;
      const int ng = (int)gmv.size();
      if (ng == 0) {
        A.ngroups = 0;
        A.gmask = nullptr;
        A.gstart = nullptr;
        GV_CUDA(launch_step(prec, A, jobs, 0, s));
        continue;
      }
      int g0 = 0;
      bool first = true;
      while (g0 < ng) {
        int g1 = g0;
        while (g1 < ng) {
          const int nt = gsv[g1 + 1] - gsv[g0];
          // real path: the group tables share the CTA with two 32 KiB (FP32 2^13 / FP64 2^12) partner tiles
          const size_t need = cplx ? xyc_smem_bytes(prec, g1 + 1 - g0, nt) : xy_smem_bytes(prec, g1 + 1 - g0, nt);
          if (need > (cplx ? 160 : 120) * 1024) break;
          ++g1;
        }
        if (g1 == g0) return fail(GVQE_EUNSUPPORTED, "X-mask group %d has too many terms", g0);
        PassArgs B = A;
        B.gmask = (cplx ? h->d_cgm : h->d_gm) + g0;
        B.gstart = (cplx ? h->d_cgs : h->d_gs) + g0;
        B.ngroups = g1 - g0;
        B.tz = cplx ? h->d_ctz : h->d_tz;
        B.tc = cplx ? h->d_ctr[prec] : tc;
        B.tci = cplx ? h->d_cti[prec] : nullptr;
        const bool last = (g1 == ng);
        B.flags = A.flags & ~(F_ENERGY | F_WRITE_LAMBDA | F_ACCUM);
        if (!first) B.flags |= F_ACCUM;
        if (last) B.flags |= (A.flags & (F_ENERGY | F_WRITE_LAMBDA));
        if (!last) B.flags |= F_WRITE_LAMBDA;
        if (!last || (A.flags & F_WRITE_LAMBDA)) {
          if (!B.out) return fail(GVQE_EUNSUPPORTED, "chunked X-mask groups need a lambda buffer");
        }
        B.lam_in = B.out;  // chunks after the first accumulate onto lambda
        const int nt = gsv[g1] - gsv[g0];
        GV_CUDA(launch_step(prec, B, jobs, nt, s));
        first = false;
        g0 = g1;
      }
    }
    if (pl->dir.empty()) continue;
    count_launches(1);
    GV_CUDA(launch_reduce(part, pl->part_stride, (const RedEntry *)pl->d_dir.ptr, pl->d_dir_count, mask ? mask + (size_t)j0 * pl->P : nullptr,
                          pl->P, E + j0, grad ? grad + (size_t)j0 * pl->P : nullptr, jobs, s));
  }
  return GVQE_OK;
}

static bool is_ham(const void *p) { return p && ((const gvqe_hamiltonian_s *)p)->magic == MAGIC_HAM; }
static bool is_ansatz(const void *p) { return p && ((const gvqe_ansatz_s *)p)->magic == MAGIC_ANSATZ; }

static int check_pair(gvqe_ansatz a, gvqe_hamiltonian h) {
  if (!is_ansatz(a)) return fail(GVQE_EINVAL, "invalid ansatz handle");
  if (!is_ham(h)) return fail(GVQE_EINVAL, "invalid Hamiltonian handle");
  if (a->n != h->n) return fail(GVQE_EINVAL, "ansatz has %d qubits but the Hamiltonian %d", a->n, h->n);
  return GVQE_OK;
}

// energies (and optionally adjoint gradients) for a batch
int gvqe::energy_impl(gvqe_ansatz a, gvqe_hamiltonian h, const double *params, const uint8_t *mask, int batch,
                      double *E, double *grad, int prec, cudaStream_t s) {
  const bool cplx = a->gates == 2;
  const bool diag = cplx ? h->cgm.empty() : h->gm.empty();
  GV_TRY(ensure_tables(h, prec, s, cplx));
  Plan *pl = get_plan(a, prec, grad != nullptr, diag);
  const int P = pl->P;
  // trig table and per-job lowest active layer
  const size_t cs_bytes = (size_t)batch * P * (prec ? 16 : 8);
  GV_TRY(a->aux.reserve(cs_bytes + (size_t)batch * 4 + 256));
  void *cs = a->aux.ptr;
  int *minlayer = (int *)((char *)a->aux.ptr + ((cs_bytes + 255) / 256) * 256);
  GV_CUDA(launch_trig(prec, params, (long long)batch * P, cs, s));
  count_launches(1);
  const int *ml = nullptr;
  if (grad) {
    GV_CUDA(launch_minlayer(mask, batch, a->n * a->gates, P, a->reps + 1, minlayer, s));
    count_launches(1);
    ml = minlayer;
  }
  return run_plan(a, h, pl, cs, mask, batch, E, grad, ml, s);
}

static int param_shift_impl(gvqe_ansatz a, gvqe_hamiltonian h, const double *params, const uint8_t *mask, int batch,
                            double *E, double *grad, int prec, cudaStream_t s) {
  const int P = a->gates * a->n * (a->reps + 1);
  std::vector<uint8_t> hmask((size_t)batch * P, 1);
  if (mask) {
    GV_CUDA(cudaMemcpyAsync(hmask.data(), mask, hmask.size(), cudaMemcpyDeviceToHost, s));
    GV_CUDA(cudaStreamSynchronize(s));
  }
  for (int b = 0; b < batch; ++b) {
    std::vector<int> act;
    for (int p = 0; p < P; ++p)
      if (hmask[(size_t)b * P + p]) act.push_back(p);
    const int rows = 2 * (int)act.size() + 1;
    GV_TRY(a->shift.reserve((size_t)rows * P * 8 + (size_t)rows * 8 + act.size() * 4 + 1024));
    double *sp = (double *)a->shift.ptr;
    double *se = sp + (size_t)rows * P;
    int *sa = (int *)(se + rows);
    if (!act.empty()) GV_CUDA(cudaMemcpyAsync(sa, act.data(), act.size() * 4, cudaMemcpyHostToDevice, s));
    GV_CUDA(launch_shift_params(params + (size_t)b * P, P, 1, sa, (int)act.size(), sp, s));
    count_launches(1);
    GV_TRY(energy_impl(a, h, sp, nullptr, rows, se, nullptr, prec, s));
    GV_CUDA(launch_shift_combine(se, P, 1, sa, (int)act.size(), E + b, grad + (size_t)b * P, s));
    count_launches(1);
    GV_CUDA(cudaStreamSynchronize(s));  // the host vector `act` and the shift buffer are reused
  }
  return GVQE_OK;
}

// ---------------------------------------------------------------- C ABI --
extern "C" {

int64_t gvqe_launch_count(void) { return (int64_t)g_launches.load(); }

int gvqe_profile_enable(int on) {
  g_err.clear();
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on != 0;
  return GVQE_OK;
}

int gvqe_profile_read(int kind, int64_t *launches, double *ms, double *bytes) {
  g_err.clear();
  if (kind < 0 || kind >= PROF_KINDS) return fail(GVQE_EINVAL, "profile kind %d", kind);
  prof_drain();
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (launches) *launches = g_prof_n[kind];
  if (ms) *ms = g_prof_ms[kind];
  if (bytes) *bytes = g_prof_bytes[kind];
  return GVQE_OK;
}

int gvqe_profile_reset(void) {
  g_err.clear();
  prof_drain();
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (int k = 0; k < PROF_KINDS; ++k) {
    g_prof_n[k] = 0;
    g_prof_ms[k] = 0;
    g_prof_bytes[k] = 0;
  }
  return GVQE_OK;
}

int gvqe_set_device_memory_limit(long long bytes) {
  g_err.clear();
  if (bytes < 0) return fail(GVQE_EINVAL, "limit %lld < 0", bytes);
  g_mem_limit = bytes;
  return GVQE_OK;
}

long long gvqe_device_memory_in_use(void) { return g_mem_used.load(); }

int gvqe_version(void) { return 10000 * GVQE_VERSION_MAJOR + 100 * GVQE_VERSION_MINOR + GVQE_VERSION_PATCH; }

const char *gvqe_last_error(void) { return g_err.c_str(); }

int gvqe_hamiltonian_create(int n_qubits, int n_terms, const char *pauli, const double *coeffs,
                            gvqe_hamiltonian *out) {
  g_err.clear();
  if (!out) return fail(GVQE_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_qubits < 1 || n_qubits > GVQE_MAX_QUBITS)
    return fail(GVQE_EINVAL, "n_qubits=%d outside [1, %d]", n_qubits, GVQE_MAX_QUBITS);
  if (n_terms < 0) return fail(GVQE_EINVAL, "n_terms=%d < 0", n_terms);
  if (n_terms > 0 && (!pauli || !coeffs)) return fail(GVQE_EINVAL, "pauli or coeffs is NULL");
  gvqe_hamiltonian_s *h = new gvqe_hamiltonian_s();
  h->magic = MAGIC_HAM;
  h->n = n_qubits;
  const int rc = parse_hamiltonian(h, n_qubits, n_terms, pauli, coeffs);
  if (rc != GVQE_OK) {
    h->magic = 0;
    delete h;
    return rc;
  }
  *out = h;
  return GVQE_OK;
}

int gvqe_hamiltonian_stats(gvqe_hamiltonian h, int *n_diag, int *n_groups, int *n_grouped, int *n_dropped) {
  g_err.clear();
  if (!is_ham(h)) return fail(GVQE_EINVAL, "invalid Hamiltonian handle");
  if (n_diag) *n_diag = (int)h->dz.size();
  if (n_groups) *n_groups = (int)h->gm.size();
  if (n_grouped) *n_grouped = h->n_grouped;
  if (n_dropped) *n_dropped = h->n_dropped;
  return GVQE_OK;
}

int gvqe_ansatz_create(int n_qubits, int reps, int entangler, gvqe_ansatz *out) {
  g_err.clear();
  if (!out) return fail(GVQE_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_qubits < 1 || n_qubits > GVQE_MAX_QUBITS)
    return fail(GVQE_EINVAL, "n_qubits=%d outside [1, %d]", n_qubits, GVQE_MAX_QUBITS);
  if (reps < 0 || reps > 64) return fail(GVQE_EINVAL, "reps=%d outside [0, 64]", reps);
  if (entangler < GVQE_ENT_LINEAR || entangler > GVQE_ENT_SCA)
    return fail(GVQE_EINVAL, "entangler %d is not one of GVQE_ENT_LINEAR .. GVQE_ENT_SCA", entangler);
  // the layer-1 gather builds the analytic product state from split tables
  for (int tb = 10; tb <= 13; ++tb) {
    int kbit;
    uint32_t hflip;
    if (!ent_l0_split(ent_map(entangler, n_qubits, 1), n_qubits, tb, &kbit, &hflip))
      return fail(GVQE_EUNSUPPORTED, "entangler %d at n=%d: layer-1 gather tables do not split", entangler,
                  n_qubits);
  }
  gvqe_ansatz_s *a = new gvqe_ansatz_s();
  a->magic = MAGIC_ANSATZ;
  a->n = n_qubits;
  a->reps = reps;
  a->ent = entangler;
  a->tile_bits = 0;
  *out = a;
  return GVQE_OK;
}

int gvqe_ansatz_set_option(gvqe_ansatz a, int option, int value) {
  g_err.clear();
  if (!is_ansatz(a)) return fail(GVQE_EINVAL, "invalid ansatz handle");
  if (option == GVQE_OPT_TILE_BITS) {
    if (value != 0 && (value < 10 || value > 13))
      return fail(GVQE_EINVAL, "tile bits %d outside [10, 13] (0 = auto)", value);
    a->tile_bits = value;
    a->tuned_tb[0] = a->tuned_tb[1] = 0;  // an explicit choice replaces a tuned one
    a->tuned_split[0] = a->tuned_split[1] = -1;
    a->tuned_xy_tb[0] = a->tuned_xy_tb[1] = 0;
    a->tune_report.clear();
    a->plans.clear();
    return GVQE_OK;
  }
  if (option == GVQE_OPT_SPLIT_PASSES) {
    if (value < SPLIT_AUTO || value > SPLIT_ALWAYS + GVQE_MAX_QUBITS)
      return fail(GVQE_EINVAL, "split mode %d is not 0 (auto), 1 (never), 2 (always) or 2 + y (y top qubits)", value);
    a->split = value;
    a->tuned_tb[0] = a->tuned_tb[1] = 0;
    a->tuned_split[0] = a->tuned_split[1] = -1;
    a->tuned_xy_tb[0] = a->tuned_xy_tb[1] = 0;
    a->tune_report.clear();
    a->plans.clear();
    return GVQE_OK;
  }
  if (option == GVQE_OPT_XY_TILE_BITS) {
    if (value != 0 && (value < 10 || value > 13))
      return fail(GVQE_EINVAL, "X-mask tile bits %d outside [10, 13] (0 = those of the first pass)", value);
    a->xy_tb = value;
    a->tuned_xy_tb[0] = a->tuned_xy_tb[1] = 0;
    a->tune_report.clear();
    a->plans.clear();
    return GVQE_OK;
  }
  if (option == GVQE_OPT_MPS_LAYERS) {
    if (value < -1 || value > MPS_MAX_LAYERS)
      return fail(GVQE_EINVAL, "closed-form layers %d outside [-1, %d] (0 = auto, -1 = none)", value, MPS_MAX_LAYERS);
    a->mps = value;
    a->plans.clear();
    return GVQE_OK;
  }
  if (option == GVQE_OPT_MPS_TENSOR) {
    if (value < -1 || value > 0)
      return fail(GVQE_EINVAL, "closed-form tensor-core mode %d is not 0 (auto) or -1 (FP32 pipe)", value);
    a->mps_tc = value;
    a->plans.clear();
    return GVQE_OK;
  }
  if (option == GVQE_OPT_GATES) {
    if (value != GVQE_GATES_RY && value != GVQE_GATES_RY_RZ)
      return fail(GVQE_EINVAL, "gate set %d is not GVQE_GATES_RY or GVQE_GATES_RY_RZ", value);
    a->gates = value;
    a->plans.clear();
    return GVQE_OK;
  }
  return fail(GVQE_EINVAL, "unknown option %d", option);
}

static int common_checks(gvqe_ansatz a, gvqe_hamiltonian h, const void *params, int batch, const void *E, int flags) {
  GV_TRY(check_pair(a, h));
  if (!params || !E) return fail(GVQE_EINVAL, "params or energies is NULL");
  if (batch < 1) return fail(GVQE_EINVAL, "batch=%d < 1", batch);
  if (flags & ~(GVQE_FP64 | GVQE_GRAD_PARAM_SHIFT)) return fail(GVQE_EINVAL, "unknown flags 0x%x", flags);
  const int prec = flags & GVQE_FP64 ? 1 : 0;
  if (eff_tile_bits(a, prec) > max_tile_bits(prec))
    return fail(GVQE_EINVAL, "tile bits %d above the %s maximum %d", eff_tile_bits(a, prec), prec ? "FP64" : "FP32",
                max_tile_bits(prec));
  return GVQE_OK;
}

int gvqe_energy(gvqe_ansatz a, gvqe_hamiltonian h, const double *params, int batch, double *energies, int flags,
                void *stream) {
  g_err.clear();
  NvtxRange range("gvqe_energy");
  GV_TRY(common_checks(a, h, params, batch, energies, flags));
  if (flags & GVQE_GRAD_PARAM_SHIFT) return fail(GVQE_EINVAL, "GVQE_GRAD_PARAM_SHIFT is a gradient flag");
  return energy_impl(a, h, params, nullptr, batch, energies, nullptr, flags & GVQE_FP64 ? 1 : 0,
                     (cudaStream_t)stream);
}

int gvqe_energy_grad(gvqe_ansatz a, gvqe_hamiltonian h, const double *params, const uint8_t *mask, int batch,
                     double *energies, double *grad, int flags, void *stream) {
  g_err.clear();
  NvtxRange range("gvqe_energy_grad");
  GV_TRY(common_checks(a, h, params, batch, energies, flags));
  if (!grad) return fail(GVQE_EINVAL, "grad is NULL");
  const int prec = flags & GVQE_FP64 ? 1 : 0;
  if (flags & GVQE_GRAD_PARAM_SHIFT)
    return param_shift_impl(a, h, params, mask, batch, energies, grad, prec, (cudaStream_t)stream);
  return energy_impl(a, h, params, mask, batch, energies, grad, prec, (cudaStream_t)stream);
}

// ----------------------------------------------------------------- readout --
static unsigned long long double_to_key(double d) {
  unsigned long long b;
  memcpy(&b, &d, sizeof(b));
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
static double key_to_double(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  double d;
  memcpy(&d, &b, sizeof(d));
  return d;
}

int gvqe_readout(gvqe_ansatz a, gvqe_hamiltonian h, const double *params, int flags, double alpha, int n_shots,
                 const double *uniforms, int64_t *shots, double *stats, int64_t *argmax, void *stream) {
  g_err.clear();
  NvtxRange range("gvqe_readout");
  if (!is_ansatz(a)) return fail(GVQE_EINVAL, "invalid ansatz handle");
  if (!params || !stats || !argmax) return fail(GVQE_EINVAL, "params, stats and argmax must be device pointers");
  if (!(alpha >= 0.0 && alpha <= 1.0)) return fail(GVQE_EINVAL, "alpha %g is outside [0, 1]", alpha);
  if (n_shots < 0 || (n_shots > 0 && (!uniforms || !shots)))
    return fail(GVQE_EINVAL, "n_shots %d needs uniforms and shots", n_shots);
  if (alpha > 0.0) GV_TRY(check_pair(a, h));
  cudaStream_t s = (cudaStream_t)stream;
  const int prec = flags & GVQE_FP64 ? 1 : 0;
  const int n = a->n;
  // the state
  Plan *pl = get_plan(a, prec, false, false, true);
  const int P = pl->P;
  GV_TRY(a->aux.reserve((size_t)P * (prec ? 16 : 8) + 256));
  GV_CUDA(launch_trig(prec, params, P, a->aux.ptr, s));
  count_launches(1);
  void *psi = nullptr;
  GV_TRY(run_plan(a, nullptr, pl, a->aux.ptr, nullptr, 1, nullptr, nullptr, nullptr, s, &psi));
  if (!psi) return fail(GVQE_EUNSUPPORTED, "the state plan kept no state");
  // workspace: chunk sums, maxima, indices, cdf, bin edges and masses, extremes, tail partials
  const long long nch = 1LL << (n - readout_chunk_bits(n));
  const int nparts = readout_tail_parts();
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t o_cmax = up(8 * nch), o_cidx = o_cmax + up(8 * nch), o_cdf = o_cidx + up(8 * nch);
  const size_t o_edges = o_cdf + up(8 * (nch + 1)), o_mass = o_edges + up(8 * (RO_BINS + 1));
  const size_t o_ext = o_mass + up(8 * RO_BINS), o_part = o_ext + up(8 * 4);
  const size_t o_es = o_part + up(8 * 3 * (size_t)nparts);  // energies at the shots
  const size_t o_mod = o_es + up(8 * (size_t)std::max(n_shots, 1));
  // complex path: the readout only needs |psi(x)|, taken once into a real array
  const size_t total_bytes = o_mod + (a->gates == 2 ? up(((size_t)1 << n) * (prec ? 8 : 4)) : 0);
  GV_TRY(a->ro.reserve(total_bytes));
  char *w = (char *)a->ro.ptr;
  if (a->gates == 2) {
    GV_CUDA(launch_ro_modulus(prec, psi, n, w + o_mod, s));
    count_launches(1);
    psi = w + o_mod;
  }
  double *csum = (double *)w, *cmax = (double *)(w + o_cmax), *cdf = (double *)(w + o_cdf);
  long long *cidx = (long long *)(w + o_cidx);
  unsigned long long *edges = (unsigned long long *)(w + o_edges);
  double *part = (double *)(w + o_part);
  unsigned long long *mass = (unsigned long long *)(w + o_mass), *ext = (unsigned long long *)(w + o_ext);
  GV_CUDA(launch_ro_prob(prec, psi, n, csum, cmax, cidx, cdf, stats, (long long *)argmax, s));
  count_launches(2);
  if (n_shots > 0) {
    GV_CUDA(launch_ro_sample(prec, psi, n, cdf, uniforms, n_shots, (long long *)shots, s));
    count_launches(1);
  }
  if (alpha == 0.0) {
    const double tail[3] = {std::nan(""), 0.0, 0.0};  // stats[1], and stats[3] = 0 passes
    GV_CUDA(cudaMemcpyAsync(stats + 1, &tail[0], sizeof(double), cudaMemcpyHostToDevice, s));
    GV_CUDA(cudaMemcpyAsync(stats + 3, &tail[1], sizeof(double), cudaMemcpyHostToDevice, s));
    GV_CUDA(cudaStreamSynchronize(s));
    return GVQE_OK;
  }
  // CVaR: the alpha-quantile tau of E under p by histogram passes, then the tail sums
  GV_TRY(ensure_tables(h, 1, s));
  const double *E = (const double *)h->T64.ptr;
  unsigned long long hext[4] = {0ull, ~0ull, 0ull, 0ull};
  std::vector<double> hedges(RO_BINS + 1);
  std::vector<unsigned long long> hkeys(RO_BINS + 1), hmass(RO_BINS);
  unsigned long long tot = 0, target = 0, below = 0;  // integer masses; below: under the current range
  double lo = 0.0, hi = 0.0, tau = 0.0;
  bool done = false, bracket = false;
  int passes = 0;
  // one histogram pass over [lo, hi) (with_outside: also the masses outside it)
  auto hist_pass = [&](bool with_outside) -> int {
    ++passes;
    const double wdt = (hi - lo) / RO_BINS;
    for (int k = 0; k < RO_BINS; ++k) hedges[k] = std::min(hi, lo + wdt * k);
    hedges[0] = lo;
    hedges[RO_BINS] = hi;
    for (int k = 1; k <= RO_BINS; ++k) hedges[k] = std::max(hedges[k], hedges[k - 1]);
    for (int k = 0; k <= RO_BINS; ++k) hkeys[k] = double_to_key(hedges[k]);
    unsigned long long z[4] = {0ull, ~0ull, 0ull, 0ull};
    GV_CUDA(cudaMemcpyAsync(edges, hkeys.data(), 8 * (RO_BINS + 1), cudaMemcpyHostToDevice, s));
    GV_CUDA(cudaMemsetAsync(mass, 0, 8 * RO_BINS, s));
    GV_CUDA(cudaMemcpyAsync(ext, z, sizeof(z), cudaMemcpyHostToDevice, s));
    GV_CUDA(launch_ro_hist(prec, psi, E, n, edges, mass, ext, with_outside ? 1 : 0, s));
    count_launches(1);
    GV_CUDA(cudaMemcpyAsync(hmass.data(), mass, 8 * RO_BINS, cudaMemcpyDeviceToHost, s));
    GV_CUDA(cudaMemcpyAsync(hext, ext, sizeof(hext), cudaMemcpyDeviceToHost, s));
    GV_CUDA(cudaStreamSynchronize(s));
    return GVQE_OK;
  };
  auto in_range_mass = [&]() {
    unsigned long long m = 0;
    for (int k = 0; k < RO_BINS; ++k) m += hmass[k];
    return m;
  };
  auto set_target = [&]() -> int {
    if (tot == 0) return fail(GVQE_EUNSUPPORTED, "the state has no probability mass");
    const double t = alpha * (double)tot;
    target = t < 1.0 ? 1ull : (unsigned long long)t;
    if (target > tot) target = tot;
    return GVQE_OK;
  };
  // A bracket from the shots' energies: their empirical alpha-quantile +- 4
  // standard errors.  One pass checks that it holds the quantile (and counts the
  // mass below and above it); otherwise the search starts from the full range.
  if (n_shots >= 256 && alpha < 1.0) {
    double *es = (double *)(w + o_es);
    GV_CUDA(launch_ro_gather(E, (const long long *)shots, n_shots, es, s));
    count_launches(1);
    std::vector<double> hes((size_t)n_shots);
    GV_CUDA(cudaMemcpyAsync(hes.data(), es, 8 * (size_t)n_shots, cudaMemcpyDeviceToHost, s));
    GV_CUDA(cudaStreamSynchronize(s));
    std::sort(hes.begin(), hes.end());
    const double K = n_shots, d = 4.0 * std::sqrt(alpha * (1.0 - alpha) / K) + 2.0 / K;
    if (alpha - d > 0.0 && alpha + d < 1.0) {
      const long long ilo = (long long)std::floor((alpha - d) * K);
      const long long ihi = std::min<long long>(n_shots - 1, (long long)std::ceil((alpha + d) * K));
      lo = hes[(size_t)ilo];
      hi = std::nextafter(hes[(size_t)ihi], HUGE_VAL);
      GV_TRY(hist_pass(true));
      tot = hext[0] + in_range_mass() + hext[3];
      GV_TRY(set_target());
      below = hext[0];
      bracket = below < target && target <= below + in_range_mass();
    }
  }
  if (!bracket) {
    const unsigned long long mm[4] = {0ull, ~0ull, 0ull, 0ull};
    GV_CUDA(cudaMemcpyAsync(ext, mm, sizeof(mm), cudaMemcpyHostToDevice, s));
    GV_CUDA(launch_ro_minmax(E, n, ext, s));
    count_launches(1);
    GV_CUDA(cudaMemcpyAsync(hext, ext, sizeof(hext), cudaMemcpyDeviceToHost, s));
    GV_CUDA(cudaStreamSynchronize(s));
    lo = key_to_double(hext[1]);
    hi = std::nextafter(key_to_double(hext[2]), HUGE_VAL);
    below = 0;
    GV_TRY(hist_pass(false));
    if (tot == 0) {
      tot = in_range_mass();
      GV_TRY(set_target());
    }
  }
  for (int pass = 0; pass < 48; ++pass) {
    if (pass > 0) GV_TRY(hist_pass(false));
    if (hext[1] == hext[2]) {  // one energy value left in the range
      tau = key_to_double(hext[1]);
      done = true;
      break;
    }
    // the first bin where the mass at or below it reaches the target (the
    // last populated bin if rounding leaves the target above the total)
    unsigned long long cum = below, at_b = below, before_last = below;
    int b = -1, lastnz = -1;
    for (int k = 0; k < RO_BINS; ++k) {
      if (hmass[k] == 0) continue;
      if (cum + hmass[k] >= target) {
        b = k;
        at_b = cum;
        break;
      }
      lastnz = k;
      before_last = cum;
      cum += hmass[k];
    }
    if (b < 0) {
      b = lastnz;
      at_b = before_last;
    }
    if (b < 0) return fail(GVQE_EUNSUPPORTED, "CVaR search lost the quantile");
    below = at_b;
    lo = hedges[b];
    hi = hedges[b + 1];
  }
  if (!done) return fail(GVQE_EUNSUPPORTED, "CVaR search did not converge");
  GV_CUDA(launch_ro_cvar(prec, psi, E, n, alpha, tau, part, stats, s));
  count_launches(2);
  const double npass = passes;
  GV_CUDA(cudaMemcpyAsync(stats + 3, &npass, sizeof(double), cudaMemcpyHostToDevice, s));
  GV_CUDA(cudaStreamSynchronize(s));
  return GVQE_OK;
}

int gvqe_entangler_inverse(int entangler, int n_qubits, int layer, const long long *y, long long *x,
                           long long count) {
  g_err.clear();
  if (entangler < GVQE_ENT_LINEAR || entangler > GVQE_ENT_SCA) return fail(GVQE_EINVAL, "entangler %d", entangler);
  if (n_qubits < 1 || n_qubits > GVQE_MAX_QUBITS) return fail(GVQE_EINVAL, "n_qubits=%d", n_qubits);
  if (layer < 1) return fail(GVQE_EINVAL, "layer=%d < 1", layer);
  if (count < 0 || (count > 0 && (!y || !x))) return fail(GVQE_EINVAL, "bad arrays");
  const EntMap e = ent_map(entangler, n_qubits, layer);
  const long long dim = 1LL << n_qubits;
  const uint32_t nmask = (uint32_t)(dim - 1);
  for (long long i = 0; i < count; ++i)
    if (y[i] < 0 || y[i] >= dim) return fail(GVQE_EINVAL, "y[%lld]=%lld outside [0, 2^%d)", i, y[i], n_qubits);
  for (long long i = 0; i < count; ++i) x[i] = (long long)ent_inv((uint32_t)y[i], nmask, e, n_qubits);
  return GVQE_OK;
}

int gvqe_plan_describe(int n_qubits, int reps, int flags, int tile_bits, char *buf, int buflen) {
  g_err.clear();
  if (n_qubits < 1 || n_qubits > GVQE_MAX_QUBITS || reps < 0 || reps > 64)
    return fail(GVQE_EINVAL, "bad size n=%d reps=%d", n_qubits, reps);
  const int prec = flags & GVQE_FP64 ? 1 : 0;
  if (tile_bits != 0 && (tile_bits < 10 || tile_bits > max_tile_bits(prec)))
    return fail(GVQE_EINVAL, "tile bits %d", tile_bits);
  Plan pl = build_plan(n_qubits, reps, prec, tile_bits, true, true);
  const std::string s = describe_plan(pl);
  if (buf && buflen > 0) {
    const size_t m = std::min<size_t>((size_t)buflen - 1, s.size());
    memcpy(buf, s.data(), m);
    buf[m] = 0;
  }
  return (int)pl.lp.size();
}

int gvqe_debug_check(void) {
  g_err.clear();
#ifndef GVQE_DEBUG
  return fail(GVQE_EUNSUPPORTED, "built without GVQE_DEBUG: no workspace guards to check");
#else
  GV_CUDA(cudaDeviceSynchronize());
  std::lock_guard<std::mutex> lk(g_guard_mu);
  std::vector<unsigned char> h(kGuard);
  for (const auto &kv : g_guarded) {
    for (int side = 0; side < 2; ++side) {
      const char *g = side ? kv.first + kv.second : kv.first - kGuard;
      GV_CUDA(cudaMemcpy(h.data(), g, kGuard, cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < kGuard; ++i)
        if (h[i] != kGuardByte)
          return fail(GVQE_ECORRUPT, "the guard %s a %zu-byte workspace was overwritten at byte %zu %s it", 
                      side ? "above" : "below", kv.second, side ? i : kGuard - i, side ? "past the end of" : "before");
    }
  }
  return GVQE_OK;
#endif
}

int gvqe_debug_poke_guard(int restore) {
  g_err.clear();
#ifndef GVQE_DEBUG
  (void)restore;
  return fail(GVQE_EUNSUPPORTED, "built without GVQE_DEBUG: no workspace guards");
#else
  std::lock_guard<std::mutex> lk(g_guard_mu);
  const std::pair<char *const, size_t> *big = nullptr;
  for (const auto &kv : g_guarded)
    if (!big || kv.second > big->second) big = &kv;
  if (!big) return fail(GVQE_EINVAL, "no live workspace");
  GV_CUDA(cudaMemset(big->first + big->second, restore ? kGuardByte : 0, 1));
  GV_CUDA(cudaDeviceSynchronize());
  return GVQE_OK;
#endif
}

int gvqe_ansatz_describe(gvqe_ansatz a, int flags, char *buf, int buflen) {
  g_err.clear();
  if (!is_ansatz(a)) return fail(GVQE_EINVAL, "invalid ansatz handle");
  if (flags & ~GVQE_FP64) return fail(GVQE_EINVAL, "flags 0x%x: only GVQE_FP32 / GVQE_FP64 apply", flags);
  const int prec = flags & GVQE_FP64 ? 1 : 0;
  if (eff_tile_bits(a, prec) > max_tile_bits(prec))
    return fail(GVQE_EINVAL, "tile bits %d too large", eff_tile_bits(a, prec));
  const Plan *pl = get_plan(a, prec, true, true);
  std::string s = describe_plan(*pl);
  if (!a->tune_report.empty()) s += a->tune_report;
  if (buf && buflen > 0) {
    const size_t m = std::min<size_t>((size_t)buflen - 1, s.size());
    memcpy(buf, s.data(), m);
    buf[m] = 0;
  }
  return (int)pl->lp.size();
}

int gvqe_destroy(void *handle) {
  g_err.clear();
  if (!handle) return GVQE_OK;
  const uint32_t magic = *(const uint32_t *)handle;
  if (magic == MAGIC_HAM) {
    cudaDeviceSynchronize();
    gvqe_hamiltonian_s *h = (gvqe_hamiltonian_s *)handle;
    h->T64.release();
    h->T32.release();
    h->G.release();
    h->magic = 0;
    delete h;
    return GVQE_OK;
  }
  if (magic == MAGIC_ANSATZ) {
    cudaDeviceSynchronize();
    gvqe_ansatz_s *a = (gvqe_ansatz_s *)handle;
    a->ws.release();
    a->aux.release();
    a->shift.release();
    a->ro.release();
    a->tune.release();
    for (auto &kv : a->plans) kv.second.d_dir.release();
    a->magic = 0;
    delete a;
    return GVQE_OK;
  }
  if (magic == MAGIC_BATCH) return batch_destroy((gvqe_batch_s *)handle);
  return fail(GVQE_EINVAL, "not a gvqe handle");
}

}  // extern "C"

// ------------------------------------------- helpers for the batch path --
int energy_one(gvqe_ansatz a, gvqe_hamiltonian h, const double *params, const uint8_t *mask, double *E, double *grad,
               int prec, cudaStream_t s) {
  return energy_impl(a, h, params, mask, 1, E, grad, prec, s);
}

int prepare_tables(gvqe_hamiltonian h, int prec, cudaStream_t s) { return ensure_tables(h, prec, s); }
