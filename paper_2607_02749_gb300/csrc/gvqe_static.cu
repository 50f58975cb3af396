// gvqe_static.cu -- gvqe_energy_static: energies without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need an
// energy: an embedding runtime that owns every cudaMalloc of the process (a
// custom allocator or a fixed memory budget that this library may not draw
// on), or a latency-critical loop where the first-call allocation of the
// regular workspaces is not acceptable.  For them this entry point evaluates
// the same energies as gvqe_energy for small registers with every scratch
// buffer (diagonal table, trig table, state vectors, partial sums, reduction
// directory) carved out of one file-scope device array of fixed size,
// GVQE_STATIC_SCRATCH_BYTES.
//
// The array lives in every GPU that loads this library until the process
// exits.  Host code cannot use the array's symbol as a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress
// (with that device current) and caches it; make that first call before any
// stream capture.  All calls share the one array and the last call's contents
// stay in it: everything that must start at zero is cleared by each call, and
// two calls whose GPU work overlaps (different streams, or different host
// threads on one device) race on the array.  Every host-to-device copy reads
// host memory owned by the two handles (the Hamiltonian's merged Z-masks and
// coefficients, the ansatz's cached energy plan), never a local of this call.
#include <cstring>
#include <mutex>
#include <vector>

#include "gvqe.h"
#include "gvqe_engine.cuh"
#include "gvqe_internal.h"

namespace gvqe {

static __device__ __align__(256) unsigned char g_static_scratch[GVQE_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_ptr[kMaxDevices] = {nullptr};

int static_scratch(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(GVQE_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(GVQE_EUNSUPPORTED, "device %d above the supported %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return fail(GVQE_ECUDA, "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return GVQE_OK;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace gvqe

using namespace gvqe;

extern "C" int gvqe_energy_static(gvqe_ansatz a, gvqe_hamiltonian h, const double *params, int batch,
                                  double *energies, int flags, void *stream) {
  g_err.clear();
  if (!a || a->magic != MAGIC_ANSATZ) return fail(GVQE_EINVAL, "invalid ansatz handle");
  if (!h || h->magic != MAGIC_HAM) return fail(GVQE_EINVAL, "invalid Hamiltonian handle");
  if (a->n != h->n) return fail(GVQE_EINVAL, "ansatz has %d qubits but the Hamiltonian %d", a->n, h->n);
  if (a->gates != 1) return fail(GVQE_EUNSUPPORTED, "gvqe_energy_static takes the RY ansatz (GVQE_GATES_RY) only");
  if (!params || !energies) return fail(GVQE_EINVAL, "params or energies is NULL");
  if (batch < 1) return fail(GVQE_EINVAL, "batch=%d < 1", batch);
  if (flags & ~GVQE_FP64) return fail(GVQE_EINVAL, "flags 0x%x: only GVQE_FP32 / GVQE_FP64 apply", flags);
  if (!h->gm.empty())
    return fail(GVQE_EUNSUPPORTED, "gvqe_energy_static takes diagonal (I/Z-only) Hamiltonians");
  const int prec = flags & GVQE_FP64 ? 1 : 0;
  if (eff_tile_bits(a, prec) > max_tile_bits(prec))
    return fail(GVQE_EINVAL, "tile bits %d too large", eff_tile_bits(a, prec));
  cudaStream_t s = (cudaStream_t)stream;

  // The energy plan (forward passes with the energy fused into the last one),
  // cached on the ansatz so that its reduction directory outlives this call.
  const Plan &pl = *get_plan(a, prec, false, true, false, false);  // no closed-form layers: no table region here
  const int n = a->n, P = pl.P;
  const size_t S = (size_t)1 << n;
  const size_t es = prec ? 8 : 4;
  const size_t ndz = h->dz.size();
  // scratch layout (256-byte aligned parts)
  size_t off = 0;
  const size_t o_t64 = off;
  off = up256(off + S * 8);
  const size_t o_t32 = off;
  if (!prec) off = up256(off + S * 4);
  const size_t o_dz = off;
  off = up256(off + ndz * 4);
  const size_t o_dc = off;
  off = up256(off + ndz * 8);
  const size_t o_cs = off;
  off = up256(off + (size_t)batch * P * 2 * es);
  const size_t o_dir = off;
  off = up256(off + pl.dir.size() * sizeof(RedEntry));
  const size_t o_part = off;
  off = up256(off + (size_t)batch * pl.part_stride * 8);
  const size_t o_bufs = off;
  off = up256(off + (size_t)pl.n_bufs * batch * S * es);
  if (off > (size_t)GVQE_STATIC_SCRATCH_BYTES)
    return fail(GVQE_EINVAL,
                "n=%d reps=%d batch=%d needs %zu bytes of static scratch; the limit is %d bytes "
                "(GVQE_STATIC_SCRATCH_BYTES): use gvqe_energy or a smaller batch",
                n, a->reps, batch, off, GVQE_STATIC_SCRATCH_BYTES);
  void *base = nullptr;
  const int rc = static_scratch(&base);
  if (rc != GVQE_OK) return rc;
  char *b = (char *)base;
  double *t64 = (double *)(b + o_t64);
  float *t32 = (float *)(b + o_t32);

#define GS_CUDA(expr)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess) return fail(GVQE_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));   \
  } while (0)

  // diagonal table E(x) = sum_z chat[z] (-1)^popcount(x & z), rebuilt in the scratch:
  // the table region starts at zero, the merged coefficients are scattered, then
  // Walsh-Hadamard passes run in place (FP64), rounded once to FP32 in FP32 mode.
  GS_CUDA(cudaMemsetAsync(t64, 0, S * 8, s));
  if (ndz > 0) {
    GS_CUDA(cudaMemcpyAsync(b + o_dz, h->dz.data(), ndz * 4, cudaMemcpyHostToDevice, s));
    GS_CUDA(cudaMemcpyAsync(b + o_dc, h->dc.data(), ndz * 8, cudaMemcpyHostToDevice, s));
    GS_CUDA(launch_scatter_coeffs((const uint32_t *)(b + o_dz), (const double *)(b + o_dc), (int)ndz, t64, s));
    count_launches(1);
    for (const LayerPass &lp : layer_passes(n, 1, 0)) {
      PassArgs A;
      memset(&A, 0, sizeof(A));
      A.kind = K_WHT;
      A.load_mode = LD_PLAIN;
      A.store_mode = ST_PLAIN;
      A.n = n;
      set_pass_layout(A, lp);
      A.tiles = 1LL << (n - lp.tb);
      A.gate_mask = lp.gmask;
      A.in = t64;
      A.out = t64;
      A.P = 1;
      GS_CUDA(launch_step(1, A, 1, 0, s));
    }
  }
  if (!prec) {
    GS_CUDA(launch_convert_table(t64, t32, (long long)S, s));
    count_launches(1);
  }

  // trig table and reduction directory
  void *cs = b + o_cs;
  GS_CUDA(launch_trig(prec, params, (long long)batch * P, cs, s));
  count_launches(1);
  GS_CUDA(cudaMemcpyAsync(b + o_dir, pl.dir.data(), pl.dir.size() * sizeof(RedEntry), cudaMemcpyHostToDevice, s));

  double *part = (double *)(b + o_part);
  char *bufs = b + o_bufs;
  auto buf_ptr = [&](int id) -> void * {
    if (id < 0) return nullptr;
    return bufs + (size_t)id * batch * S * es;
  };
  for (const PassStep &st : pl.steps) {
    PassArgs A = st.A;
    A.job0 = 0;
    A.cs = cs;
    A.table = prec ? (const void *)t64 : (const void *)t32;
    A.in = buf_ptr(st.in);
    A.in_stride = (long long)S;
    A.lam_in = buf_ptr(st.lam);
    A.lam_stride = (long long)S;
    A.out = buf_ptr(st.out);
    A.out_stride = (long long)S;
    A.part = part + (st.part_region >= 0 ? st.part_region : 0);
    A.epart = part + (st.epart_region >= 0 ? st.epart_region : 0);
    A.part_stride = pl.part_stride;
    A.minlayer = nullptr;
    GS_CUDA(launch_step(prec, A, batch, 0, s));
  }
  GS_CUDA(launch_reduce(part, pl.part_stride, (const RedEntry *)(b + o_dir), (int)pl.dir.size(), nullptr, P,
                        energies, nullptr, batch, s));
  count_launches(1);
#undef GS_CUDA
  return GVQE_OK;
}
