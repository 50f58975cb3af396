// gvqe_internal.h -- host-side handle and plan structures of the gvqe library.
#pragma once
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "gvqe_engine.cuh"

#define GVQE_VERSION_MAJOR 0
#define GVQE_VERSION_MINOR 1
#define GVQE_VERSION_PATCH 0

namespace gvqe {

enum : uint32_t {
  MAGIC_HAM = 0x47564831u,     // "GVH1"
  MAGIC_ANSATZ = 0x47564131u,  // "GVA1"
  MAGIC_BATCH = 0x47564231u,   // "GVB1"
};

int fail(int code, const char *fmt, ...);
extern thread_local std::string g_err;

// An owned device allocation that only grows.
struct DevBuf {
  void *ptr = nullptr;
  size_t bytes = 0;
  int reserve(size_t need);
  void release();
};

// One pass of an RY layer: tile bits [0,c) -> global [0,c), [c,tb) -> global [a, a+tb-c)
// or, split, [c, c+k1) -> [a, a+k1) and [c+k1, tb) -> [a+k1+gap, a+gap+tb-c);
// gates on the tile bits in gmask.
struct LayerPass {
  int c, a, tb;
  uint32_t gmask;
  int k1 = 0, gap = 0;
};

// Strided-pass layout choice (GVQE_OPT_SPLIT_PASSES).
enum SplitMode : int { SPLIT_AUTO = 0, SPLIT_NEVER = 1, SPLIT_ALWAYS = 2 };

// One launch of a plan.  Buffer ids index the plan's state buffers (-1 = none).
struct PassStep {
  PassArgs A;
  int in = -1, lam = -1, out = -1;
  long long part_region = -1, epart_region = -1;
  bool xy = false;
};

struct Plan {
  int n = 0, reps = 0, prec = 0, P = 0, tile_bits = 0;
  std::vector<LayerPass> lp;
  std::vector<PassStep> steps;
  int n_bufs = 0, n_states = 0;
  long long state_elems = 0;
  long long part_stride = 0;  // doubles of partial sums per job
  std::map<int, RedEntry> param_dir;
  std::vector<RedEntry> dir;  // energy entry first, then one per parameter
  int final_buf = -1;         // state-only plans: buffer of the final state
  int mps_layers = 0;         // leading layers written in closed form (K_MPS steps)
  bool mps_grad = false;      // ... and their gradients from lambda and the matrix product
  bool mps_tc = false;        // ... with the bond-16 chunk contractions on the tensor cores
  long long mps_elems = 0;    // floats of closed-form tables per job (one stage at a time)
  DevBuf d_dir;
  int d_dir_count = 0;
};

std::vector<LayerPass> layer_passes(int n, int prec, int tile_bits, int split = SPLIT_AUTO);
void set_pass_layout(PassArgs &A, const LayerPass &lp);
void count_launches(int k);
// tile_grad_l0: lay the layer-0 gradient partials out per tile (one CTA of
// tile bits per partial), as the persistent batch kernel computes them,
// instead of per warp of the standalone layer-0 gradient pass.
// state_only: the forward passes alone, the final state kept (Plan::final_buf).
// gates: 1 = RY layers (real amplitudes), 2 = full EfficientSU2 layers, RY then
// RZ on every qubit (complex amplitudes; diagonal H, energy and gradient only).
// xy_tb: tile bits of the X-mask pass (0: those of the layer's first pass).
// mps_layers: the leading layers after layer 0 whose states K_MPS steps write
// in closed form (0: none; see mps_layers_for).  mps_tc: at bond dimension 16
// the writer and the gradient pass over lambda contract on the tensor cores (F_MPS_TC).
Plan build_plan(int n, int reps, int prec, int tile_bits, bool want_grad, bool diag, bool tile_grad_l0 = false,
                bool state_only = false, int ent = ENT_LINEAR, int gates = 1, int split = SPLIT_AUTO, int xy_tb = 0,
                int mps_layers = 0, bool mps_tc = true);
// How many leading layers a plan may write in closed form: FP32, RY layers,
// an entangler whose index map ties each qubit only to the one below it
// (linear, full, reverse linear), n >= MPS_MIN_QUBITS, and never the last
// layer (which carries the energy epilogue); `want` is GVQE_OPT_MPS_LAYERS
// (0 = up to MPS_AUTO_LAYERS, -1 = none, 1..MPS_MAX_LAYERS = at most that many).
int mps_layers_for(int n, int reps, int prec, int ent, int gates, int want);
// Kernels one closed-form step launches (the high-qubit gradient tree, from n = 28, takes two).
int mps_step_kernels(const PassArgs &A);
std::string describe_plan(const Plan &pl);
// One tile-pass launch, counted by gvqe_launch_count and timed by the event
// profiler when it is on.
cudaError_t launch_step(int prec, const PassArgs &A, int jobs, int nterm, cudaStream_t s);

}  // namespace gvqe

struct gvqe_hamiltonian_s {
  uint32_t magic = 0;
  int n = 0;
  // diagonal part: unique z-masks with merged coefficients (the all-I string has z = 0)
  std::vector<uint32_t> dz;
  std::vector<double> dc;
  // X-mask groups (m != 0, even number of Y): group g owns terms [gs[g], gs[g+1])
  std::vector<uint32_t> gm;
  std::vector<int> gs;
  std::vector<uint32_t> tz;
  std::vector<double> tc;
  int n_grouped = 0, n_dropped = 0;
  // the complex path's X-mask groups: every string with X/Y letters, odd #Y
  // included, with real and imaginary coefficient parts (i^#Y folded in)
  std::vector<uint32_t> cgm;
  std::vector<int> cgs;
  std::vector<uint32_t> ctz;
  std::vector<double> ctr, cti;
  gvqe::DevBuf CG;
  uint32_t *d_cgm = nullptr;
  int *d_cgs = nullptr;
  uint32_t *d_ctz = nullptr;
  void *d_ctr[2] = {nullptr, nullptr}, *d_cti[2] = {nullptr, nullptr};  // FP32, FP64
  double abs_sum = 0.0;
  gvqe::DevBuf T64, T32, G;
  gvqe::DevBuf TC[2];  // complex path: each table entry twice (re/im), FP32 and FP64
  uint32_t *d_gm = nullptr;
  int *d_gs = nullptr;
  uint32_t *d_tz = nullptr;
  double *d_tc64 = nullptr;
  float *d_tc32 = nullptr;
};

struct gvqe_ansatz_s {
  uint32_t magic = 0;
  int n = 0, reps = 0, ent = 0;
  int gates = 1;  // 1: RY layers; 2: RY then RZ (the complex path)
  int tile_bits = 0;  // 0 = automatic (GVQE_OPT_TILE_BITS, both precisions)
  int split = 0;      // gvqe::SplitMode (GVQE_OPT_SPLIT_PASSES, both precisions)
  // per precision (FP32, FP64): the plan gvqe_autotune chose (0 / -1: none), which
  // takes the place of tile_bits / split for that precision until an option is set
  int tuned_tb[2] = {0, 0};
  int tuned_split[2] = {-1, -1};
  int xy_tb = 0;                 // GVQE_OPT_XY_TILE_BITS (0: the first pass's tile bits)
  int tuned_xy_tb[2] = {0, 0};   // per precision, chosen by gvqe_autotune (0: none)
  int mps = 0;                   // GVQE_OPT_MPS_LAYERS (0 auto, -1 none, 1..4 at most that many)
  int mps_tc = 0;                // GVQE_OPT_MPS_TENSOR (0 auto = tensor cores, -1 = FP32 pipe)
  std::map<int, gvqe::Plan> plans;
  gvqe::DevBuf ws, aux, shift, ro, tune;
  std::string tune_report;  // the last gvqe_autotune sweep and its choice (empty: not tuned)
};

struct gvqe_batch_s;
int batch_destroy(gvqe_batch_s *b);

namespace gvqe {
// The tile bits and strided layout an ansatz's plans take in one precision.
inline int eff_tile_bits(const gvqe_ansatz_s *a, int prec) { return a->tuned_tb[prec] ? a->tuned_tb[prec] : a->tile_bits; }
inline int eff_split(const gvqe_ansatz_s *a, int prec) { return a->tuned_split[prec] >= 0 ? a->tuned_split[prec] : a->split; }
inline int eff_xy_tb(const gvqe_ansatz_s *a, int prec) { return a->tuned_xy_tb[prec] ? a->tuned_xy_tb[prec] : a->xy_tb; }
// The ansatz's cached plan for (precision, gradient or not, diagonal H or not,
// state only); it and its host-side reduction directory live until the
// ansatz is destroyed or one of its options changes.
// allow_mps = false: no closed-form layers (callers without a table region).
Plan *get_plan(gvqe_ansatz_s *a, int prec, bool want_grad, bool diag, bool state_only = false, bool allow_mps = true);
// Energies (and adjoint gradients when grad != NULL) of a batch: the body of
// gvqe_energy / gvqe_energy_grad after their argument checks.
int energy_impl(gvqe_ansatz_s *a, gvqe_hamiltonian_s *h, const double *params, const uint8_t *mask, int batch,
                double *E, double *grad, int prec, cudaStream_t s);
}  // namespace gvqe
