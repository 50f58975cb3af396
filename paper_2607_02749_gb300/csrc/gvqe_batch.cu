// gvqe_batch.cu -- many independent restricted-update problems (Section IV-D,
// Eq. 11) in one persistent kernel launch, replayed from a CUDA graph.
//
// Work items are (instance, step, tile) triples.  Each instance's steps are:
// PREP (cos/sin of its parameters, lowest active layer of its mask), the tile
// passes of its plan (forward, backward, layer-0 gradient), and REDUCE (its
// energy and gradient from the partial sums).  CTAs claim items from one
// global ticket counter in a fixed stage-major order (every instance's step s
// before any instance's step s + 1).  An item waits, with a bounded spin, until
// every tile of the previous step of its own instance has finished.  A wait only
// ever targets items with smaller tickets, which were claimed earlier by CTAs
// that are running, so the smallest unfinished item can always proceed: the
// schedule cannot deadlock, whatever the number of resident CTAs.  A wait that
// outlives its budget sets an error word, skips its work and still signals
// completion; the host reports GVQE_ETIMEOUT.
//
// Producers publish with __threadfence() + atomicAdd on the step's counter;
// consumers spin on an acquire load, then every state load goes through L2.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "gvqe.h"
#include "gvqe_internal.h"
#include "gvqe_tile.cuh"

namespace gvqe {

enum StepKind : int { S_PREP = 0, S_PASS = 1, S_REDUCE = 2 };
constexpr int SEG_BLK_BITS = 6;  // tickets per entry of the segment index: 64

struct BatchStep {
  PassArgs A;        // pass arguments with this instance's buffers (job 0 of one)
  int kind;          // StepKind
  int inst;          // instance index
  int dep;           // step this one waits for (-1: none)
  unsigned dep_need; // completions of `dep` required (its item count)
  unsigned items;    // items of this step
  const RedEntry *dir;  // REDUCE: directory of the instance
  int ndir;
  int n, reps;       // PREP: register size and repetitions
};

struct BatchIO {
  const double *params;  // P doubles
  const uint8_t *mask;   // P bytes or NULL (all active)
  double *grad;          // P doubles or NULL
  double *energy;        // one double
};

struct BatchArgs {
  const BatchStep *steps;
  const unsigned *seg_start;  // first ticket of each step in schedule order
  const int *seg_step;        // step index of each segment
  const int *blk_seg;         // segment holding ticket (b << SEG_BLK_BITS), per block b of tickets
  int nseg;
  unsigned total;
  unsigned *ticket;
  unsigned *done;             // completions per step (+ spare counters)
  int *err;
  const BatchIO *io;
  long long timeout_cycles;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <typename T>
__device__ void batch_prep(const BatchStep &st, const BatchIO &io) {
  using T2 = typename V2<T>::type;
  const PassArgs &A = st.A;
  T2 *cs = reinterpret_cast<T2 *>(const_cast<void *>(A.cs));
  for (int p = threadIdx.x; p < A.P; p += blockDim.x) {
    double s, c;
    sincos(0.5 * io.params[p], &s, &c);
    T2 v;
    v.x = (T)c;
    v.y = (T)s;
    cs[p] = v;
  }
  if (threadIdx.x == 0) {
    int m = st.reps + 1;  // nothing active: no backward pass needed
    if (io.mask == nullptr) {
      m = 0;
    } else {
      for (int p = 0; p < A.P; ++p)
        if (io.mask[p]) {
          m = p / st.n;
          break;
        }
    }
    *const_cast<int *>(A.minlayer) = m;
  }
}

__device__ void batch_reduce(const BatchStep &st, const BatchIO &io) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double *part = st.A.part;
  for (int e = wid; e < st.ndir; e += nw) {
    const RedEntry d = st.dir[e];
    double s = 0.0;
    for (int i = lane; i < d.count; i += 32) s += __ldcg(part + d.off + i);
    s = warp_sum(s);
    if (lane == 0) {
      if (d.param < 0) {
        *io.energy = s;
      } else if (io.grad != nullptr) {
        const bool on = io.mask == nullptr || io.mask[d.param] != 0;
        io.grad[d.param] = on ? s : 0.0;
      }
    }
  }
}

template <typename T, int TB>
__device__ void batch_pass(const PassArgs &A, uint32_t tile) {
  const bool full = A.c >= TB;
  switch (A.kind) {
    case K_FWD:
      if (!full) {
        fwd_tile<T, TB, false, LD_PLAIN, false>(A, 0, tile);
      } else {
        switch (A.load_mode) {
          case LD_PLAIN: fwd_tile<T, TB, true, LD_PLAIN, false>(A, 0, tile); break;
          case LD_GATHER: fwd_tile<T, TB, true, LD_GATHER, false>(A, 0, tile); break;
          case LD_L0_GATHER: fwd_tile<T, TB, true, LD_L0_GATHER, false>(A, 0, tile); break;
          default: fwd_tile<T, TB, true, LD_L0, false>(A, 0, tile); break;
        }
      }
      break;
    case K_BWD:
      if (full)
        bwd_tile<T, TB, true>(A, 0, tile);
      else
        bwd_tile<T, TB, false>(A, 0, tile);
      break;
    case K_GRAD_L0:
      grad_l0_tile<T, TB>(A, 0, tile);
      break;
    default:
      break;
  }
}

// Bring the inputs of one future item into L2 (a hint: no data is waited for or
// kept).  Forward passes that gather through the entangler or start from the
// analytic product state are left out; the others read their tile as rows of
// 2^c contiguous amplitudes (a whole 2^TB run in layout FULL).
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

template <typename T, int TB>
__device__ void batch_prefetch(const BatchStep &st, unsigned tile) {
  if (st.kind != S_PASS) return;
  const PassArgs &A = st.A;
  if (A.kind == K_FWD && A.load_mode != LD_PLAIN) return;
  const T *src[2] = {nullptr, nullptr};
  if (A.kind == K_FWD) {
    src[0] = reinterpret_cast<const T *>(A.in);
  } else if (A.kind == K_BWD) {
    src[0] = reinterpret_cast<const T *>(A.in);
    src[1] = reinterpret_cast<const T *>((A.flags & F_LAMBDA_INIT) ? A.table : A.lam_in);
  } else if (A.kind == K_GRAD_L0) {
    src[0] = reinterpret_cast<const T *>(A.lam_in);
  } else {
    return;
  }
  const bool full = A.c >= TB;
  const uint32_t base = (A.kind == K_GRAD_L0) ? (tile << TB) : tile_base(tile_of_block(tile, (uint32_t)A.tiles, A.pair_mask), A, TB);
  constexpr int LINE = 128 / (int)sizeof(T);  // amplitudes per 128-byte line
  const int run = full ? (1 << TB) : (1 << A.c);
  const int lines_per_run = run > LINE ? run / LINE : 1;
  const int step = run > LINE ? LINE : run;
  const int nlines = (1 << TB) / step;
  for (int i = threadIdx.x; i < nlines; i += blockDim.x) {
    const uint32_t r = (uint32_t)(i / lines_per_run), l = (uint32_t)(i % lines_per_run);
    const uint32_t off = full ? base + (uint32_t)i * LINE : base + tile_goff(r << A.c, A) + l * LINE;
    prefetch_l2(src[0] + off);
    if (src[1]) prefetch_l2(src[1] + off);
  }
}

// Thread 0 of each CTA holds two claimed tickets besides the current item: the
// next item's inputs are prefetched into L2 while the current one runs, and the
// ticket after it is claimed then (the atomic's latency hides behind the item's
// work).  A CTA always finishes the smallest ticket it holds first, so the
// smallest unfinished item is always being run by the CTA that claimed it and
// its dependencies (smaller tickets) are finished: the schedule still cannot
// deadlock.
template <typename T, int TB>
__global__ void __launch_bounds__(1 << (TB - 5), sizeof(T) == 8 ? 2 : (TB == 12 ? 5 : (TB == 11 ? 8 : 16)))
k_batch(const BatchArgs B) {
  __shared__ unsigned s_tile, s_ntile;
  __shared__ int s_si, s_nsi, s_ok;
  // thread 0: seg lookup of a ticket (segment index, from the block index, forward)
  auto lookup = [&](unsigned item, int *si, unsigned *tile) {
    int lo = B.blk_seg[item >> SEG_BLK_BITS];
    while (lo + 1 < B.nseg && B.seg_start[lo + 1] <= item) ++lo;
    *si = B.seg_step[lo];
    *tile = item - B.seg_start[lo];
  };
  unsigned nxt = 0, nxt2 = 0;  // claimed tickets after the current one (thread 0)
  int cur_si = -1, nxt_si = -1;
  unsigned cur_tile = 0, nxt_tile = 0;
  if (threadIdx.x == 0) {
    const unsigned first = atomicAdd(B.ticket, 1u);
    nxt = atomicAdd(B.ticket, 1u);
    if (first < B.total) lookup(first, &cur_si, &cur_tile);
  }
  for (;;) {
    if (threadIdx.x == 0) {
      if (cur_si >= 0) {
        nxt_si = -1;
        if (nxt < B.total) {
          nxt2 = atomicAdd(B.ticket, 1u);
          lookup(nxt, &nxt_si, &nxt_tile);
        }
        const BatchStep &st = B.steps[cur_si];
        int ok = 1;
        if (st.dep >= 0 && ld_acquire(B.done + st.dep) < st.dep_need) {
          const long long t0 = clock64();
          while (ld_acquire(B.done + st.dep) < st.dep_need) {
            if (clock64() - t0 > B.timeout_cycles) {
              atomicOr(B.err, 1);
              ok = 0;
              break;
            }
            __nanosleep(128);
          }
        }
        s_ok = ok;
        s_tile = cur_tile;
        s_nsi = nxt_si;
        s_ntile = nxt_tile;
      }
      s_si = cur_si;
    }
    __syncthreads();
    const int si = s_si;
    if (si < 0) break;
    const unsigned tile = s_tile;
    const BatchStep &st = B.steps[si];
    if (s_nsi >= 0) batch_prefetch<T, TB>(B.steps[s_nsi], s_ntile);
    if (s_ok) {
      const BatchIO io = B.io[st.inst];
      if (st.kind == S_PREP)
        batch_prep<T>(st, io);
      else if (st.kind == S_REDUCE)
        batch_reduce(st, io);
      else
        batch_pass<T, TB>(st.A, tile);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(B.done + (si), 1u);
      cur_si = nxt_si;
      cur_tile = nxt_tile;
      nxt = nxt2;
    }
  }
}

// The staged schedule: instances with the same plan (n, reps, entangler,
// layout) form a group, and a group runs its plan's steps as launches in order
// on a stream of its own (one branch of the batch's graph; the branches run
// side by side).  A launch covers one step of every instance of the group: CTA
// (x, y) runs tile x of the step of the group's y-th instance.  The stream order
// takes the place of the persistent kernel's waits, and no CTA searches for its
// work item.
template <typename T, int TB>
__global__ void __launch_bounds__(1 << (TB - 5), sizeof(T) == 8 ? 2 : 5) k_stage(const BatchArgs B, const int *ids) {
  const BatchStep &st = B.steps[ids[blockIdx.y]];
  if (st.kind == S_PREP) {
    batch_prep<T>(st, B.io[st.inst]);
  } else if (st.kind == S_REDUCE) {
    batch_reduce(st, B.io[st.inst]);
  } else {
    batch_pass<T, TB>(st.A, blockIdx.x);
  }
}

// ------------------------------------------------------------------- host --
// (the dynamic shared-memory limit is raised by batch_occupancy before capture)
template <typename T, int TB>
static cudaError_t launch_batch(const BatchArgs &B, int ctas, size_t smem, cudaStream_t s) {
  k_batch<T, TB><<<ctas, 1 << (TB - 5), smem, s>>>(B);
  return cudaGetLastError();
}

template <typename T, int TB>
static cudaError_t launch_stage(const BatchArgs &B, const int *ids, unsigned tiles, unsigned insts, size_t smem,
                                cudaStream_t s) {
  const cudaError_t e = cudaFuncSetAttribute(k_stage<T, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_stage<T, TB><<<dim3(tiles, insts), 1 << (TB - 5), smem, s>>>(B, ids);
  return cudaGetLastError();
}

template <typename T, int TB>
static int batch_occupancy(size_t smem) {
  int per = 0;
  cudaFuncSetAttribute(k_batch<T, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch<T, TB>, 1 << (TB - 5), smem) != cudaSuccess)
    per = 1;
  return std::max(1, per);
}

}  // namespace gvqe

using namespace gvqe;

// Live bytes per wave of the batch schedule (GVQE_BATCH_OPT_WAVE_BYTES, 0: one
// wave); gvqe_batch_autotune picks among 0 and budgets sized so that a wave's
// pass inputs and outputs fit the 129 MB L2.
constexpr long long kDefaultWaveBytes = 0;

// One compiled schedule (energy-only or energy + gradient).
struct BatchSchedule {
  bool built = false;
  DevBuf dev;  // steps, segments, counters, io, workspace
  BatchArgs args{};
  int ctas = 0;
  size_t smem = 0;
  std::vector<Plan> plans;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int nsteps = 0;
  int counters = 0;
  int waves = 0;
  int groups = 0;  // staged schedule: groups of instances that share one plan
};

struct gvqe_batch_s {
  uint32_t magic = 0;
  int prec = 0;
  bool persistent = false;
  long long wave_bytes = kDefaultWaveBytes;  // GVQE_BATCH_OPT_WAVE_BYTES
  int schedule = GVQE_BATCH_STAGED;         // GVQE_BATCH_OPT_SCHEDULE
  int tile_bits = 12;                        // GVQE_BATCH_OPT_TILE_BITS (FP64: always 12)
  std::string tune_report;
  // instances of the persistent launch (slot k -> instance pidx[k]) and the
  // ones evaluated by single calls in the same run (n < 12, X/Y strings, RY+RZ)
  std::vector<int> pidx, sidx;
  std::vector<gvqe_ansatz> a;
  std::vector<gvqe_hamiltonian> h;
  BatchSchedule sched[2];  // [0] energies only, [1] energies + gradients
  std::vector<BatchIO> io_host;
  bool io_valid[2] = {false, false};
};

namespace {

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// 2^12-amplitude tiles in both precisions: an item is one tile, and in FP32 five
// 128-thread CTAs per SM (96 registers) keep more items in flight than two
// 256-thread CTAs on 2^13 tiles (measured for the 256-instance cluster batch:
// 4.97 ms on 2^13 tiles, 4.78 ms at four CTAs of 2^12, 4.48 ms at five).
int tile_bits_for(const gvqe_batch_s *b) { return b->tile_bits; }

// Launch of the persistent kernel for the batch's tile size: 2^12 (four warps
// per CTA), 2^11 (two) or 2^10 (one warp per CTA, so every block barrier of
// the tile rounds is a warp barrier and each warp claims its own items).
cudaError_t launch_batch_tb(int prec, int tb, const BatchArgs &B, int ctas, size_t smem, cudaStream_t s) {
  if (prec) return launch_batch<double, 12>(B, ctas, smem, s);
  switch (tb) {
    case 10: return launch_batch<float, 10>(B, ctas, smem, s);
    case 11: return launch_batch<float, 11>(B, ctas, smem, s);
    default: return launch_batch<float, 12>(B, ctas, smem, s);
  }
}
cudaError_t launch_stage_tb(int prec, int tb, const BatchArgs &B, const int *ids, unsigned tiles, unsigned insts,
                            size_t smem, cudaStream_t s) {
  if (prec) return launch_stage<double, 12>(B, ids, tiles, insts, smem, s);
  switch (tb) {
    case 10: return launch_stage<float, 10>(B, ids, tiles, insts, smem, s);
    case 11: return launch_stage<float, 11>(B, ids, tiles, insts, smem, s);
    default: return launch_stage<float, 12>(B, ids, tiles, insts, smem, s);
  }
}
int batch_occupancy_tb(int prec, int tb, size_t smem) {
  if (prec) return batch_occupancy<double, 12>(smem);
  switch (tb) {
    case 10: return batch_occupancy<float, 10>(smem);
    case 11: return batch_occupancy<float, 11>(smem);
    default: return batch_occupancy<float, 12>(smem);
  }
}

long long wait_budget_cycles() {
  // bounded device-side waits: GVQE_WAIT_TIMEOUT_MS (default 2000 ms) at ~2 GHz
  long long ms = 2000;
  if (const char *e = getenv("GVQE_WAIT_TIMEOUT_MS")) ms = std::max(1LL, atoll(e));
  return ms * 2000000LL;
}

#define GB_CUDA(expr)                                                                         \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess) return fail(GVQE_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));  \
  } while (0)

int build_grouped(gvqe_batch_s *b, int want_grad);

int build_schedule(gvqe_batch_s *b, int want_grad) {
  if (b->schedule == GVQE_BATCH_STAGED) return build_grouped(b, want_grad);
  BatchSchedule &sc = b->sched[want_grad];
  const int prec = b->prec;
  const int TB = tile_bits_for(b);
  const size_t es = prec ? 8 : 4;
  const int ni = (int)b->pidx.size();  // slots of the persistent launch
  auto A_of = [&](int k) { return b->a[b->pidx[k]]; };
  auto H_of = [&](int k) { return b->h[b->pidx[k]]; };
  sc.plans.clear();
  sc.plans.reserve(ni);
  for (int i = 0; i < ni; ++i)
    sc.plans.push_back(build_plan(A_of(i)->n, A_of(i)->reps, prec, TB, want_grad != 0, true, true, false, A_of(i)->ent, 1,
                                  eff_split(A_of(i), prec)));

  // device layout: [steps][seg_start][seg_step][counters][io][per-instance workspace]
  std::vector<BatchStep> steps;
  std::vector<std::vector<int>> inst_steps(ni);
  for (int i = 0; i < ni; ++i) {
    const Plan &pl = sc.plans[i];
    BatchStep prep{};
    prep.kind = S_PREP;
    prep.inst = i;
    prep.items = 1;
    prep.n = pl.n;
    prep.reps = pl.reps;
    inst_steps[i].push_back((int)steps.size());
    steps.push_back(prep);
    for (const PassStep &ps : pl.steps) {
      BatchStep st{};
      st.kind = S_PASS;
      st.inst = i;
      st.A = ps.A;
      st.items = (unsigned)ps.A.tiles;
      inst_steps[i].push_back((int)steps.size());
      steps.push_back(st);
    }
    BatchStep red{};
    red.kind = S_REDUCE;
    red.inst = i;
    red.items = 1;
    red.ndir = (int)pl.dir.size();
    inst_steps[i].push_back((int)steps.size());
    steps.push_back(red);
  }
  const int nsteps = (int)steps.size();
  for (int i = 0; i < ni; ++i)
    for (size_t k = 1; k < inst_steps[i].size(); ++k) {
      BatchStep &st = steps[inst_steps[i][k]];
      st.dep = inst_steps[i][k - 1];
      st.dep_need = steps[st.dep].items;
    }
  // host-injected fault for tests: the first pass of instance 0 waits on a counter nothing signals
  const bool inject = getenv("GVQE_TEST_UNSATISFIABLE_WAIT") != nullptr;
  if (inject && inst_steps[0].size() > 1) {
    BatchStep &st = steps[inst_steps[0][1]];
    st.dep = nsteps;  // a spare counter
    st.dep_need = 1;
  }
  // Ticket order: the instances, larger first, cut into waves whose live bytes
  // add up to at most wave_bytes (one wave when 0), and inside each wave
  // stage-major (every instance's step s before any instance's step s + 1).  A
  // wave's states are written and read again while they are still in L2; the
  // next wave's first items need nothing from it and fill the GPU as it drains.
  std::vector<int> order(ni);
  for (int i = 0; i < ni; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return A_of(x)->n > A_of(y)->n; });
  // an instance's live bytes while one of its passes runs: the pass input, its
  // output and (backward) the stored forward state or the table
  auto inst_bytes = [&](int i) { return (size_t)3 * sc.plans[i].state_elems * es; };
  std::vector<std::vector<int>> waves;
  size_t wave_sum = 0;
  for (int i : order) {
    const size_t bi = inst_bytes(i);
    if (waves.empty() || (b->wave_bytes > 0 && wave_sum + bi > (size_t)b->wave_bytes && !waves.back().empty())) {
      waves.emplace_back();
      wave_sum = 0;
    }
    waves.back().push_back(i);
    wave_sum += bi;
  }
  std::vector<unsigned> seg_start;
  std::vector<int> seg_step;
  unsigned tick = 0;
  for (const std::vector<int> &wv : waves) {
    size_t max_stage = 0;
    for (int i : wv) max_stage = std::max(max_stage, inst_steps[i].size());
    for (size_t s = 0; s < max_stage; ++s) {
      for (int i : wv) {
        if (s >= inst_steps[i].size()) continue;
        const int si = inst_steps[i][s];
        seg_start.push_back(tick);
        seg_step.push_back(si);
        tick += steps[si].items;
      }
    }
  }
  sc.waves = (int)waves.size();
  const int nseg = (int)seg_start.size();
  const int counters = nsteps + 1;
  // segment index: for each block of 2^SEG_BLK_BITS tickets, the segment holding its first ticket
  const unsigned nblk = (tick >> SEG_BLK_BITS) + 1;
  std::vector<int> blk_seg(nblk);
  {
    int sg = 0;
    for (unsigned bk = 0; bk < nblk; ++bk) {
      const unsigned first = bk << SEG_BLK_BITS;
      while (sg + 1 < nseg && seg_start[sg + 1] <= first) ++sg;
      blk_seg[bk] = sg;
    }
  }

  // workspace offsets
  size_t off = 0;
  const size_t o_steps = off;
  off = up256(off + sizeof(BatchStep) * nsteps);
  const size_t o_segs = off;
  off = up256(off + sizeof(unsigned) * nseg);
  const size_t o_segstep = off;
  off = up256(off + sizeof(int) * nseg);
  const size_t o_blkseg = off;
  off = up256(off + sizeof(int) * nblk);

  const size_t o_ctr = off;  // ticket, err, done[counters]
  off = up256(off + sizeof(unsigned) * (2 + counters));
  const size_t o_io = off;
  off = up256(off + sizeof(BatchIO) * ni);
  const size_t o_dir = off;
  size_t dir_total = 0;
  for (int i = 0; i < ni; ++i) dir_total += sc.plans[i].dir.size();
  off = up256(off + sizeof(RedEntry) * dir_total);
  std::vector<size_t> o_inst(ni);
  for (int i = 0; i < ni; ++i) {
    const Plan &pl = sc.plans[i];
    o_inst[i] = off;
    off = up256(off + (size_t)pl.P * 2 * es);                   // cs
    off = up256(off + sizeof(int));                              // minlayer
    off = up256(off + (size_t)pl.part_stride * 8);               // partials
    off = up256(off + (size_t)pl.n_bufs * pl.state_elems * es);  // state buffers
  }
  {
    const int rc = sc.dev.reserve(off);
    if (rc != GVQE_OK) return rc;
  }
  char *base = (char *)sc.dev.ptr;
  // resolve the pointers of every step
  size_t dir_off = 0;
  for (int i = 0; i < ni; ++i) {
    const Plan &pl = sc.plans[i];
    char *ib = base + o_inst[i];
    void *cs = ib;
    char *p = ib + up256((size_t)pl.P * 2 * es);
    int *ml = (int *)p;
    p += 256;
    double *part = (double *)p;
    p += up256((size_t)pl.part_stride * 8);
    char *bufs = p;
    auto buf = [&](int id) -> void * { return id < 0 ? nullptr : bufs + (size_t)id * pl.state_elems * es; };
    const void *table = prec ? H_of(i)->T64.ptr : H_of(i)->T32.ptr;
    const RedEntry *dir = (const RedEntry *)(base + o_dir) + dir_off;
    for (size_t k = 0; k < inst_steps[i].size(); ++k) {
      BatchStep &st = steps[inst_steps[i][k]];
      st.A.cs = cs;
      st.A.minlayer = ml;
      st.A.P = pl.P;
      st.A.part = part;
      st.A.part_stride = pl.part_stride;
      if (st.kind == S_PASS) {
        const PassStep &ps = pl.steps[k - 1];
        st.A.job0 = 0;
        st.A.table = table;
        st.A.in = buf(ps.in);
        st.A.in_stride = pl.state_elems;
        st.A.lam_in = buf(ps.lam);
        st.A.lam_stride = pl.state_elems;
        st.A.out = buf(ps.out);
        st.A.out_stride = pl.state_elems;
        st.A.part = part + (ps.part_region >= 0 ? ps.part_region : 0);
        st.A.epart = part + (ps.epart_region >= 0 ? ps.epart_region : 0);
      } else if (st.kind == S_REDUCE) {
        st.dir = dir;
      }
    }
    dir_off += pl.dir.size();
  }
  std::vector<RedEntry> dirs;
  dirs.reserve(dir_total);
  for (int i = 0; i < ni; ++i) dirs.insert(dirs.end(), sc.plans[i].dir.begin(), sc.plans[i].dir.end());
  GB_CUDA(cudaMemcpy(base + o_steps, steps.data(), sizeof(BatchStep) * nsteps, cudaMemcpyHostToDevice));
  GB_CUDA(cudaMemcpy(base + o_segs, seg_start.data(), sizeof(unsigned) * nseg, cudaMemcpyHostToDevice));
  GB_CUDA(cudaMemcpy(base + o_segstep, seg_step.data(), sizeof(int) * nseg, cudaMemcpyHostToDevice));
  GB_CUDA(cudaMemcpy(base + o_blkseg, blk_seg.data(), sizeof(int) * nblk, cudaMemcpyHostToDevice));

  if (!dirs.empty()) GB_CUDA(cudaMemcpy(base + o_dir, dirs.data(), sizeof(RedEntry) * dirs.size(), cudaMemcpyHostToDevice));

  BatchArgs &B = sc.args;
  B.steps = (const BatchStep *)(base + o_steps);
  B.seg_start = (const unsigned *)(base + o_segs);
  B.seg_step = (const int *)(base + o_segstep);
  B.blk_seg = (const int *)(base + o_blkseg);
  B.nseg = nseg;
  B.total = tick;
  B.ticket = (unsigned *)(base + o_ctr);
  B.err = (int *)(base + o_ctr + sizeof(unsigned));
  B.done = (unsigned *)(base + o_ctr + 2 * sizeof(unsigned));
  B.io = (const BatchIO *)(base + o_io);
  B.timeout_cycles = wait_budget_cycles();
  sc.nsteps = nsteps;
  sc.counters = counters;
  // one CTA's shared memory: the largest of a forward tile and a backward tile (psi + lambda)
  sc.smem = 2 * (es << TB);
  int sms = 1, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per = batch_occupancy_tb(prec, TB, sc.smem);
  sc.ctas = std::max(1, sms * per);

  // the graph: clear ticket, error word and counters, then the persistent launch
  cudaStream_t cap;
  GB_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemsetAsync(base + o_ctr, 0, sizeof(unsigned) * (2 + counters), cap);
    const cudaError_t le = launch_batch_tb(prec, TB, B, sc.ctas, sc.smem, cap);
    e = cudaStreamEndCapture(cap, &sc.graph);
    if (e == cudaSuccess) e = le;
  }
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) return fail(GVQE_ECUDA, "batch graph capture: %s", cudaGetErrorString(e));
  GB_CUDA(cudaGraphInstantiate(&sc.exec, sc.graph, 0));
  sc.built = true;
  b->io_valid[want_grad] = false;
  return GVQE_OK;
}

int batch_loop(gvqe_batch_s *b, const double *const *params, const uint8_t *const *masks, double *energies,
               double *const *grads, cudaStream_t s);

// The staged schedule.  Instances with the same plan (n, reps, entangler, strided
// layout) form a group of J jobs whose states, partial sums, trig tables and
// diagonal tables (copied from each Hamiltonian) sit job after job, so each of
// the plan's passes runs as ONE launch of the regular pass kernels over all J
// jobs (the persistent, prefetching backward included), as gvqe_energy_grad
// runs a batch of parameter vectors.  Per group, on a branch of its own of the
// graph: a PREP launch (one CTA per job: its cos/sin table and lowest active
// layer), the plan's passes, and a REDUCE launch (one CTA per job: its energy
// and gradient into the caller's buffers).  The branches run side by side.
int build_grouped(gvqe_batch_s *b, int want_grad) {
  BatchSchedule &sc = b->sched[want_grad];
  const int prec = b->prec;
  const size_t es = prec ? 8 : 4;
  const int tbg = max_tile_bits(prec);
  const int ni = (int)b->pidx.size();
  auto A_of = [&](int k) { return b->a[b->pidx[k]]; };
  auto H_of = [&](int k) { return b->h[b->pidx[k]]; };
  std::map<std::vector<int>, std::vector<int>> by_plan;  // plan key -> slots
  for (int k = 0; k < ni; ++k)
    by_plan[{A_of(k)->n, A_of(k)->reps, A_of(k)->ent, eff_split(A_of(k), prec)}].push_back(k);
  struct Group {
    std::vector<int> slots;
    Plan plan;
    size_t o_cs, o_ml, o_part, o_tab, o_bufs, o_dir;
  };
  std::vector<Group> groups;
  std::vector<BatchStep> steps;  // PREP then REDUCE per slot
  size_t off = 0;
  const size_t o_steps = off;
  off = up256(off + sizeof(BatchStep) * 2 * (size_t)ni);
  const size_t o_ids = off;
  off = up256(off + sizeof(int) * 2 * (size_t)ni);
  const size_t o_ctr = off;  // ticket, err (unused here, kept zero for the error check)
  off = up256(off + sizeof(unsigned) * 2);
  const size_t o_io = off;
  off = up256(off + sizeof(BatchIO) * ni);
  for (auto &kv : by_plan) {
    Group g;
    g.slots = kv.second;
    const gvqe_ansatz a0 = A_of(g.slots[0]);
    g.plan = build_plan(a0->n, a0->reps, prec, tbg, want_grad != 0, true, false, false, a0->ent, 1,
                        eff_split(a0, prec));
    const size_t J = g.slots.size(), S = (size_t)g.plan.state_elems;
    g.o_cs = off;
    off = up256(off + J * g.plan.P * 2 * es);
    g.o_ml = off;
    off = up256(off + J * 4);
    g.o_part = off;
    off = up256(off + J * (size_t)g.plan.part_stride * 8);
    g.o_tab = off;
    off = up256(off + J * S * es);
    g.o_bufs = off;
    off = up256(off + (size_t)g.plan.n_bufs * J * S * es);
    g.o_dir = off;
    off = up256(off + sizeof(RedEntry) * std::max<size_t>(1, g.plan.dir.size()));
    groups.push_back(std::move(g));
  }
  // larger groups first: their longer chains of passes start early
  std::stable_sort(groups.begin(), groups.end(), [](const Group &x, const Group &y) {
    return x.slots.size() * (size_t)x.plan.state_elems * x.plan.steps.size() >
           y.slots.size() * (size_t)y.plan.state_elems * y.plan.steps.size();
  });
  {
    const int rc = sc.dev.reserve(off);
    if (rc != GVQE_OK) return rc;
  }
  char *base = (char *)sc.dev.ptr;
  std::vector<int> prep_ids(ni), red_ids(ni);
  steps.resize(2 * (size_t)ni);
  for (const Group &g : groups) {
    const size_t S = (size_t)g.plan.state_elems;
    for (size_t j = 0; j < g.slots.size(); ++j) {
      const int k = g.slots[j];
      BatchStep &pr = steps[2 * (size_t)k];
      pr = BatchStep{};
      pr.kind = S_PREP;
      pr.inst = k;
      pr.items = 1;
      pr.dep = -1;
      pr.n = g.plan.n;
      pr.reps = g.plan.reps;
      pr.A.P = g.plan.P;
      pr.A.cs = base + g.o_cs + j * g.plan.P * 2 * es;
      pr.A.minlayer = (const int *)(base + g.o_ml) + j;
      BatchStep &rd = steps[2 * (size_t)k + 1];
      rd = BatchStep{};
      rd.kind = S_REDUCE;
      rd.inst = k;
      rd.items = 1;
      rd.dep = -1;
      rd.A.part = (double *)(base + g.o_part) + j * (size_t)g.plan.part_stride;
      rd.dir = (const RedEntry *)(base + g.o_dir);
      rd.ndir = (int)g.plan.dir.size();
      // this job's diagonal table
      const gvqe_hamiltonian h = H_of(k);
      GB_CUDA(cudaMemcpy(base + g.o_tab + j * S * es, prec ? h->T64.ptr : h->T32.ptr, S * es, cudaMemcpyDeviceToDevice));
    }
    if (!g.plan.dir.empty())
      GB_CUDA(cudaMemcpy(base + g.o_dir, g.plan.dir.data(), sizeof(RedEntry) * g.plan.dir.size(), cudaMemcpyHostToDevice));
  }
  // PREP and REDUCE ids in group order (a launch covers one group's contiguous range)
  std::vector<int> ids;
  for (const Group &g : groups)
    for (int k : g.slots) ids.push_back(2 * k);
  for (const Group &g : groups)
    for (int k : g.slots) ids.push_back(2 * k + 1);
  GB_CUDA(cudaMemcpy(base + o_steps, steps.data(), sizeof(BatchStep) * steps.size(), cudaMemcpyHostToDevice));
  GB_CUDA(cudaMemcpy(base + o_ids, ids.data(), sizeof(int) * ids.size(), cudaMemcpyHostToDevice));
  GB_CUDA(cudaMemset(base + o_ctr, 0, sizeof(unsigned) * 2));

  BatchArgs &B = sc.args;
  B = BatchArgs{};
  B.steps = (const BatchStep *)(base + o_steps);
  B.ticket = (unsigned *)(base + o_ctr);
  B.err = (int *)(base + o_ctr + sizeof(unsigned));
  B.io = (const BatchIO *)(base + o_io);
  sc.smem = 0;
  sc.groups = (int)groups.size();
  const int *d_ids = (const int *)(base + o_ids);

  cudaStream_t cap;
  GB_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  cudaError_t le = cudaSuccess;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> evs;
  // waves of groups (GVQE_BATCH_OPT_WAVE_BYTES: live bytes, three states per job):
  // the groups of a wave run side by side, a wave starts when the previous ends
  std::vector<size_t> wave_start = {0};
  {
    size_t sum = 0;
    for (size_t gi = 0; gi < groups.size(); ++gi) {
      const size_t live = (size_t)3 * groups[gi].slots.size() * (size_t)groups[gi].plan.state_elems * es;
      if (b->wave_bytes > 0 && gi > wave_start.back() && sum + live > (size_t)b->wave_bytes) {
        wave_start.push_back(gi);
        sum = 0;
      }
      sum += live;
    }
    wave_start.push_back(groups.size());
  }
  sc.waves = (int)wave_start.size() - 1;
  if (e == cudaSuccess) {
    cudaEvent_t fork = nullptr;
    size_t first = 0;
    for (size_t gi = 0; gi < groups.size() && le == cudaSuccess; ++gi) {
      if (std::find(wave_start.begin(), wave_start.end(), gi) != wave_start.end()) {
        fork = nullptr;  // a new wave forks from the capture stream after the last one joined
        le = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        if (le != cudaSuccess) break;
        evs.push_back(fork);
        le = cudaEventRecord(fork, cap);
        if (le != cudaSuccess) break;
      }
      const Group &g = groups[gi];
      const int J = (int)g.slots.size();
      const size_t S = (size_t)g.plan.state_elems;
      cudaStream_t gs = nullptr;
      le = cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking);
      if (le != cudaSuccess) break;
      streams.push_back(gs);
      le = cudaStreamWaitEvent(gs, fork, 0);
      if (le == cudaSuccess) le = launch_stage_tb(prec, 12, B, d_ids + first, 1, (unsigned)J, 0, gs);
      char *bufs = base + g.o_bufs;
      for (const PassStep &st : g.plan.steps) {
        if (le != cudaSuccess) break;
        PassArgs A = st.A;
        A.job0 = 0;
        A.cs = base + g.o_cs;
        A.table = base + g.o_tab;
        A.table_stride = (long long)S;
        A.in = st.in < 0 ? nullptr : bufs + (size_t)st.in * J * S * es;
        A.in_stride = (long long)S;
        A.lam_in = st.lam < 0 ? nullptr : bufs + (size_t)st.lam * J * S * es;
        A.lam_stride = (long long)S;
        A.out = st.out < 0 ? nullptr : bufs + (size_t)st.out * J * S * es;
        A.out_stride = (long long)S;
        double *part = (double *)(base + g.o_part);
        A.part = part + (st.part_region >= 0 ? st.part_region : 0);
        A.epart = part + (st.epart_region >= 0 ? st.epart_region : 0);
        A.part_stride = g.plan.part_stride;
        A.minlayer = (const int *)(base + g.o_ml);
        le = launch_pass(prec, A, J, 0, gs);
      }
      if (le == cudaSuccess) le = launch_stage_tb(prec, 12, B, d_ids + ni + first, 1, (unsigned)J, 0, gs);
      cudaEvent_t join = nullptr;
      if (le == cudaSuccess) le = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
      if (le == cudaSuccess) {
        evs.push_back(join);
        le = cudaEventRecord(join, gs);
      }
      if (le == cudaSuccess) le = cudaStreamWaitEvent(cap, join, 0);
      first += (size_t)J;
    }
    e = cudaStreamEndCapture(cap, &sc.graph);
    if (e == cudaSuccess) e = le;
  }
  for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
  for (cudaStream_t gs : streams) cudaStreamDestroy(gs);
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) return fail(GVQE_ECUDA, "batch graph capture (staged): %s", cudaGetErrorString(e));
  GB_CUDA(cudaGraphInstantiate(&sc.exec, sc.graph, 0));
  sc.built = true;
  b->io_valid[want_grad] = false;
  return GVQE_OK;
}

}  // namespace

int batch_destroy(gvqe_batch_s *b) {
  cudaDeviceSynchronize();
  for (BatchSchedule &sc : b->sched) {
    if (sc.exec) cudaGraphExecDestroy(sc.exec);
    if (sc.graph) cudaGraphDestroy(sc.graph);
    sc.dev.release();
  }
  b->magic = 0;
  delete b;
  return GVQE_OK;
}

// energy / gradient of one instance through the regular path (gvqe_api.cu)
int energy_one(gvqe_ansatz a, gvqe_hamiltonian h, const double *params, const uint8_t *mask, double *E, double *grad,
               int prec, cudaStream_t s);
int prepare_tables(gvqe_hamiltonian h, int prec, cudaStream_t s);

namespace {
// Which instances the persistent kernel takes: RY layers, a diagonal Hamiltonian
// and n at least the batch tile bits; the others are evaluated by single calls.
void classify(gvqe_batch_s *b) {
  b->pidx.clear();
  b->sidx.clear();
  for (size_t i = 0; i < b->a.size(); ++i) {
    const gvqe_ansatz a = b->a[i];
    const gvqe_hamiltonian h = b->h[i];
    const bool small = b->schedule != GVQE_BATCH_STAGED && a->n < tile_bits_for(b);
    if (small || !h->gm.empty() || a->gates != 1)
      b->sidx.push_back((int)i);
    else
      b->pidx.push_back((int)i);
  }
  b->persistent = !b->pidx.empty();
}

int batch_loop(gvqe_batch_s *b, const double *const *params, const uint8_t *const *masks, double *energies,
               double *const *grads, cudaStream_t s) {
  for (int i : b->sidx) {
    const int rc = energy_one(b->a[i], b->h[i], params[i], masks ? masks[i] : nullptr, energies + i,
                              grads ? grads[i] : nullptr, b->prec, s);
    if (rc != GVQE_OK) return rc;
  }
  return GVQE_OK;
}
}  // namespace

extern "C" {

int gvqe_batch_create(int n_inst, const gvqe_ansatz *ansatze, const gvqe_hamiltonian *hams, int flags,
                      gvqe_batch *out) {
  g_err.clear();
  if (!out) return fail(GVQE_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_inst < 1 || !ansatze || !hams) return fail(GVQE_EINVAL, "n_inst=%d or NULL instance arrays", n_inst);
  if (flags & ~GVQE_FP64) return fail(GVQE_EINVAL, "unknown flags 0x%x", flags);
  const int prec = flags & GVQE_FP64 ? 1 : 0;
  for (int i = 0; i < n_inst; ++i) {
    gvqe_ansatz a = ansatze[i];
    gvqe_hamiltonian h = hams[i];
    if (!a || a->magic != MAGIC_ANSATZ) return fail(GVQE_EINVAL, "instance %d: invalid ansatz handle", i);
    if (!h || h->magic != MAGIC_HAM) return fail(GVQE_EINVAL, "instance %d: invalid Hamiltonian handle", i);
    if (a->n != h->n) return fail(GVQE_EINVAL, "instance %d: ansatz has %d qubits, Hamiltonian %d", i, a->n, h->n);
  }
  for (int i = 0; i < n_inst; ++i) {
    const int rc = prepare_tables(hams[i], prec, nullptr);
    if (rc != GVQE_OK) return rc;
  }
  gvqe_batch_s *b = new gvqe_batch_s();
  b->magic = MAGIC_BATCH;
  b->prec = prec;
  b->a.assign(ansatze, ansatze + n_inst);
  b->h.assign(hams, hams + n_inst);
  classify(b);
  *out = b;
  return GVQE_OK;
}

int gvqe_batch_set_option(gvqe_batch b, int option, long long value) {
  g_err.clear();
  if (!b || b->magic != MAGIC_BATCH) return fail(GVQE_EINVAL, "invalid batch handle");
  if (option == GVQE_BATCH_OPT_WAVE_BYTES) {
    if (value < 0) return fail(GVQE_EINVAL, "wave bytes %lld < 0", value);
    if (value == b->wave_bytes) return GVQE_OK;
  } else if (option == GVQE_BATCH_OPT_SCHEDULE) {
    if (value != GVQE_BATCH_PERSISTENT && value != GVQE_BATCH_STAGED)
      return fail(GVQE_EINVAL, "batch schedule %lld is not GVQE_BATCH_PERSISTENT or GVQE_BATCH_STAGED", value);
    if (value == b->schedule) return GVQE_OK;
  } else if (option == GVQE_BATCH_OPT_TILE_BITS) {
    if (value < 10 || value > 12) return fail(GVQE_EINVAL, "batch tile bits %lld outside [10, 12]", value);
    if (b->prec && value != 12) return fail(GVQE_EUNSUPPORTED, "FP64 batches run 2^12-amplitude tiles only");
    if (value == b->tile_bits) return GVQE_OK;
  } else {
    return fail(GVQE_EINVAL, "unknown batch option %d", option);
  }
  cudaDeviceSynchronize();
  if (option == GVQE_BATCH_OPT_WAVE_BYTES) {
    b->wave_bytes = value;
  } else if (option == GVQE_BATCH_OPT_SCHEDULE) {
    b->schedule = (int)value;
    classify(b);
  } else {
    b->tile_bits = (int)value;
    classify(b);
  }
  for (BatchSchedule &sc : b->sched) {  // rebuilt (and recaptured) on the next run
    if (sc.exec) cudaGraphExecDestroy(sc.exec);
    if (sc.graph) cudaGraphDestroy(sc.graph);
    sc.exec = nullptr;
    sc.graph = nullptr;
    sc.built = false;
  }
  b->io_valid[0] = b->io_valid[1] = false;
  return GVQE_OK;
}

int gvqe_batch_run(gvqe_batch b, const double *const *params, const uint8_t *const *masks, double *energies,
                   double *const *grads, void *stream);

int gvqe_batch_autotune(gvqe_batch b, const double *const *params, const uint8_t *const *masks, double *energies,
                        double *const *grads, char *report, int report_len, void *stream) {
  g_err.clear();
  if (!b || b->magic != MAGIC_BATCH) return fail(GVQE_EINVAL, "invalid batch handle");
  std::string rep;
  auto put = [&]() {
    if (report && report_len > 0) {
      const size_t m = std::min<size_t>((size_t)report_len - 1, rep.size());
      memcpy(report, rep.data(), m);
      report[m] = 0;
    }
  };
  if (!b->persistent) {
    rep = "batch autotune: instance by instance (no persistent schedule to tune)\n";
    put();
    return GVQE_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  struct Cand {
    int sched, tb;
    long long wb;
  };
  std::vector<Cand> cands;
  for (int tb : {12, 11, 10}) {
    if (b->prec && tb != 12) continue;
    cands.push_back({GVQE_BATCH_PERSISTENT, tb, 0});
  }
  cands.push_back({GVQE_BATCH_PERSISTENT, 12, 256ll << 20});
  for (long long wb : {0ll, 128ll << 20, 256ll << 20})  // the regular plans' tiles (2^13 FP32, 2^12 FP64)
    cands.push_back({GVQE_BATCH_STAGED, 12, wb});
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  GB_CUDA(cudaEventCreate(&e0));
  GB_CUDA(cudaEventCreate(&e1));
  const long long keep = b->wave_bytes;
  const int keep_tb = b->tile_bits, keep_sched = b->schedule;
  Cand best{-1, -1, 0};
  double best_ms = 0.0;
  std::string sweep;
  int rc = GVQE_OK;
  for (const Cand &cd : cands) {
    rc = gvqe_batch_set_option(b, GVQE_BATCH_OPT_SCHEDULE, cd.sched);
    if (rc == GVQE_OK) rc = gvqe_batch_set_option(b, GVQE_BATCH_OPT_TILE_BITS, cd.tb);
    if (rc == GVQE_OK) rc = gvqe_batch_set_option(b, GVQE_BATCH_OPT_WAVE_BYTES, cd.wb);
    if (rc == GVQE_OK) rc = gvqe_batch_run(b, params, masks, energies, grads, stream);  // build + warm
    if (rc != GVQE_OK) break;
    const int timed = 3;
    cudaEventRecord(e0, s);
    for (int r = 0; r < timed && rc == GVQE_OK; ++r) rc = gvqe_batch_run(b, params, masks, energies, grads, stream);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    if (rc != GVQE_OK) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double per = ms / timed;
    const int g = grads ? 1 : 0;
    char line[200];
    if (cd.sched == GVQE_BATCH_STAGED)
      snprintf(line, sizeof(line), "%sstaged wave=%lldMiB (%d plan groups in %d waves, %zu of %zu instances in it): %.3f ms",
               sweep.empty() ? "" : "; ", cd.wb >> 20, b->sched[g].groups, b->sched[g].waves, b->pidx.size(),
               b->a.size(), per);
    else
      snprintf(line, sizeof(line), "%spersistent tiles=2^%d wave=%lldMiB (%d waves, %zu of %zu instances in it): %.3f ms",
               sweep.empty() ? "" : "; ", cd.tb, cd.wb >> 20, b->sched[g].waves, b->pidx.size(), b->a.size(), per);
    sweep += line;
    if (best.tb < 0 || per < best_ms) {
      best = cd;
      best_ms = per;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != GVQE_OK) {
    gvqe_batch_set_option(b, GVQE_BATCH_OPT_SCHEDULE, keep_sched);
    gvqe_batch_set_option(b, GVQE_BATCH_OPT_TILE_BITS, keep_tb);
    gvqe_batch_set_option(b, GVQE_BATCH_OPT_WAVE_BYTES, keep);
    return rc;
  }
  rc = gvqe_batch_set_option(b, GVQE_BATCH_OPT_SCHEDULE, best.sched);
  if (rc == GVQE_OK) rc = gvqe_batch_set_option(b, GVQE_BATCH_OPT_TILE_BITS, best.tb);
  if (rc == GVQE_OK) rc = gvqe_batch_set_option(b, GVQE_BATCH_OPT_WAVE_BYTES, best.wb);
  if (rc != GVQE_OK) return rc;
  char line[200];
  if (best.sched == GVQE_BATCH_STAGED)
    snprintf(line, sizeof(line),
             "batch autotune: staged schedule (plan groups, regular pass kernels), wave bytes %lld MiB, %.3f ms per run\n",
             best.wb >> 20, best_ms);
  else
    snprintf(line, sizeof(line),
             "batch autotune: persistent schedule, tiles 2^%d, wave bytes %lld MiB (%s), %.3f ms per run\n", best.tb,
             best.wb >> 20, best.wb == 0 ? "one wave" : "waves", best_ms);
  rep = std::string(line) + "batch autotune sweep: " + sweep + "\n";
  b->tune_report = rep;
  put();
  return GVQE_OK;
}

int gvqe_batch_run(gvqe_batch b, const double *const *params, const uint8_t *const *masks, double *energies,
                   double *const *grads, void *stream) {
  g_err.clear();
  if (!b || b->magic != MAGIC_BATCH) return fail(GVQE_EINVAL, "invalid batch handle");
  if (!params || !energies) return fail(GVQE_EINVAL, "params or energies is NULL");
  const size_t ni = b->a.size();
  for (size_t i = 0; i < ni; ++i) {
    if (!params[i]) return fail(GVQE_EINVAL, "params[%zu] is NULL", i);
    if (grads && !grads[i]) return fail(GVQE_EINVAL, "grads[%zu] is NULL", i);
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (!b->persistent) return batch_loop(b, params, masks, energies, grads, s);
  const int g = grads ? 1 : 0;
  BatchSchedule &sc = b->sched[g];
  if (!sc.built) {
    const int rc = build_schedule(b, g);
    if (rc != GVQE_OK) return rc;
  }
  const size_t np = b->pidx.size();
  std::vector<BatchIO> io(np);
  for (size_t k = 0; k < np; ++k) {
    const int i = b->pidx[k];
    io[k].params = params[i];
    io[k].mask = masks ? masks[i] : nullptr;
    io[k].grad = grads ? grads[i] : nullptr;
    io[k].energy = energies + i;
  }
  if (!b->io_valid[g] || b->io_host.size() != np || memcmp(io.data(), b->io_host.data(), sizeof(BatchIO) * np) != 0) {
    GB_CUDA(cudaMemcpyAsync((void *)sc.args.io, io.data(), sizeof(BatchIO) * np, cudaMemcpyHostToDevice, s));
    b->io_host = io;
    b->io_valid[g] = true;
    b->io_valid[1 - g] = false;
  }
  GB_CUDA(cudaGraphLaunch(sc.exec, s));
  count_launches(1);
  // the instances outside the persistent launch, on the same stream after it
  if (!b->sidx.empty()) {
    const int rc = batch_loop(b, params, masks, energies, grads, s);
    if (rc != GVQE_OK) return rc;
  }
  GB_CUDA(cudaStreamSynchronize(s));
  int err = 0;
  GB_CUDA(cudaMemcpy(&err, sc.args.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) return fail(GVQE_ETIMEOUT, "a bounded device-side wait of the batch kernel ran out (error word %d)", err);
  return GVQE_OK;
}

}  // extern "C"
