// gvqe_tune.cu -- the autotuner of an ansatz's tile plan and its persistent cache.
//
// The cost of one evaluation depends on how the RY layers are cut into tile
// passes: the tile size 2^k (how many qubits the contiguous first pass takes,
// how many gates each strided pass carries, how many passes a layer needs and
// how many CTAs share an SM) and the strided layout (one run of qubits per
// pass, or a low and a top run so that no tile spans more 2 MiB pages than
// needed).  The best cut differs with the register size, the precision, the
// gate set, the entangler and the batch, so gvqe_autotune measures it: every
// distinct plan among tile bits 10 .. the precision's maximum and the two
// strided layouts runs the requested evaluation (energy, or energy and adjoint
// gradient) on the caller's parameters, timed with CUDA events on the caller's
// stream, and the fastest becomes the ansatz's plan.
//
// Winners are kept in a JSON file, one entry per key (GPU name, n, reps,
// entangler, gate set, precision, gradient or not, diagonal H or not, batch):
//   {"<key>": {"tile_bits": 13, "split": 1, "ms": 312.5, "sweep": "..."}, ...}
// A later call with the same key takes the cached plan without timing.  The
// file is a cache only: deleting it, or a file that cannot be read or parsed,
// just means the sweep runs again (and the file is rewritten whole).
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include <unistd.h>

#include "gvqe.h"
#include "gvqe_engine.cuh"
#include "gvqe_internal.h"

namespace gvqe {
namespace {

struct TuneEntry {
  int tile_bits = 0;
  int split = 0;
  int xy_tb = 0;  // X-mask pass tile bits (0: the first pass's); optional in the file
  double ms = 0.0;
  std::string sweep;
};

std::mutex g_cache_mu;  // one writer of a cache file per process at a time

// ---- a small JSON reader for the cache's shape: an object of objects whose
// values are numbers or strings.  Anything else makes the whole file invalid.
struct JsonIn {
  const std::string &s;
  size_t i = 0;
  explicit JsonIn(const std::string &x) : s(x) {}
  void ws() {
    while (i < s.size() && (s[i] == ' ' || s[i] == '\t' || s[i] == '\n' || s[i] == '\r')) ++i;
  }
  bool eat(char c) {
    ws();
    if (i < s.size() && s[i] == c) {
      ++i;
      return true;
    }
    return false;
  }
  bool str(std::string *out) {
    ws();
    if (i >= s.size() || s[i] != '"') return false;
    ++i;
    out->clear();
    while (i < s.size() && s[i] != '"') {
      char c = s[i++];
      if (c == '\\') {
        if (i >= s.size()) return false;
        const char e = s[i++];
        switch (e) {
          case '"': c = '"'; break;
          case '\\': c = '\\'; break;
          case '/': c = '/'; break;
          case 'n': c = '\n'; break;
          case 't': c = '\t'; break;
          case 'r': c = '\r'; break;
          default: return false;  // \u escapes and others are never written by this file
        }
      }
      out->push_back(c);
    }
    if (i >= s.size()) return false;
    ++i;  // closing quote
    return true;
  }
  bool num(double *out) {
    ws();
    const char *b = s.c_str() + i;
    char *e = nullptr;
    const double v = strtod(b, &e);
    if (e == b) return false;
    i += (size_t)(e - b);
    *out = v;
    return true;
  }
};

bool parse_entry(JsonIn &in, TuneEntry *t) {
  if (!in.eat('{')) return false;
  bool have_tb = false, have_split = false;
  if (in.eat('}')) return false;
  for (;;) {
    std::string k;
    if (!in.str(&k) || !in.eat(':')) return false;
    in.ws();
    if (in.i < in.s.size() && in.s[in.i] == '"') {
      std::string v;
      if (!in.str(&v)) return false;
      if (k == "sweep") t->sweep = v;
    } else {
      double v = 0;
      if (!in.num(&v)) return false;
      if (k == "tile_bits") {
        t->tile_bits = (int)v;
        have_tb = true;
      } else if (k == "split") {
        t->split = (int)v;
        have_split = true;
      } else if (k == "ms") {
        t->ms = v;
      } else if (k == "xy_tile_bits") {
        t->xy_tb = (int)v;
      }
    }
    if (in.eat(',')) continue;
    if (in.eat('}')) break;
    return false;
  }
  return have_tb && have_split;
}

// The whole file, or false (then the caller treats the cache as empty).
bool parse_cache(const std::string &text, std::map<std::string, TuneEntry> *out) {
  out->clear();
  JsonIn in(text);
  if (!in.eat('{')) return false;
  if (in.eat('}')) {
    in.ws();
    return in.i == text.size();
  }
  for (;;) {
    std::string key;
    TuneEntry t;
    if (!in.str(&key) || !in.eat(':') || !parse_entry(in, &t)) return false;
    (*out)[key] = t;
    if (in.eat(',')) continue;
    if (in.eat('}')) break;
    return false;
  }
  in.ws();
  return in.i == text.size();
}

std::string json_str(const std::string &v) {
  std::string o = "\"";
  for (char c : v) {
    switch (c) {
      case '"': o += "\\\""; break;
      case '\\': o += "\\\\"; break;
      case '\n': o += "\\n"; break;
      case '\t': o += "\\t"; break;
      case '\r': o += "\\r"; break;
      default: o.push_back((unsigned char)c < 32 ? ' ' : c);
    }
  }
  return o + "\"";
}

std::string write_cache(const std::map<std::string, TuneEntry> &m) {
  std::string o = "{\n";
  bool first = true;
  char num[64];
  for (const auto &kv : m) {
    if (!first) o += ",\n";
    first = false;
    snprintf(num, sizeof(num), "%.6g", kv.second.ms);
    o += "  " + json_str(kv.first) + ": {\"tile_bits\": " + std::to_string(kv.second.tile_bits) +
         ", \"split\": " + std::to_string(kv.second.split) +
         (kv.second.xy_tb ? ", \"xy_tile_bits\": " + std::to_string(kv.second.xy_tb) : std::string()) +
         ", \"ms\": " + num +
         ", \"sweep\": " + json_str(kv.second.sweep) + "}";
  }
  return o + "\n}\n";
}

bool read_file(const char *path, std::string *out) {
  FILE *f = fopen(path, "rb");
  if (!f) return false;
  out->clear();
  char buf[4096];
  size_t k;
  while ((k = fread(buf, 1, sizeof(buf), f)) > 0) out->append(buf, k);
  fclose(f);
  return true;
}

int cache_lookup(const char *path, const std::string &key, TuneEntry *t) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  std::string text;
  if (!read_file(path, &text)) return 0;
  std::map<std::string, TuneEntry> m;
  if (!parse_cache(text, &m)) return 0;
  auto it = m.find(key);
  if (it == m.end()) return 0;
  *t = it->second;
  return 1;
}

int cache_store(const char *path, const std::string &key, const TuneEntry &t) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  std::string text;
  std::map<std::string, TuneEntry> m;
  if (read_file(path, &text) && !parse_cache(text, &m)) m.clear();  // an invalid file is rewritten
  m[key] = t;
  const std::string out = write_cache(m);
  // a writer-private temporary (processes tuning at once each rename a whole file)
  const std::string tmp = std::string(path) + ".tmp" + std::to_string((long long)getpid());
  FILE *f = fopen(tmp.c_str(), "wb");
  if (!f) return fail(GVQE_EINVAL, "cannot write the tuning cache %s", tmp.c_str());
  const bool ok = fwrite(out.data(), 1, out.size(), f) == out.size();
  fclose(f);
  if (!ok || rename(tmp.c_str(), path) != 0) {
    remove(tmp.c_str());
    return fail(GVQE_EINVAL, "cannot replace the tuning cache %s", path);
  }
  return GVQE_OK;
}

std::string split_name(int s) {
  if (s == SPLIT_NEVER) return "one run";
  if (s == SPLIT_ALWAYS) return "split";
  if (s > SPLIT_ALWAYS) return "split y=" + std::to_string(s - SPLIT_ALWAYS);
  return "auto";
}

}  // namespace
}  // namespace gvqe

using namespace gvqe;

#define GT_CUDA(expr)                                                                         \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess) return fail(GVQE_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));  \
  } while (0)

namespace {

void put_report(const std::string &r, char *buf, int buflen) {
  if (buf && buflen > 0) {
    const size_t m = std::min<size_t>((size_t)buflen - 1, r.size());
    memcpy(buf, r.data(), m);
    buf[m] = 0;
  }
}

// Events destroyed on every return path.
struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

}  // namespace

extern "C" {

int gvqe_tune_cache_get(const char *path, const char *key, int *tile_bits, int *split, double *ms) {
  g_err.clear();
  if (!path || !key || !tile_bits || !split) return fail(GVQE_EINVAL, "path, key, tile_bits or split is NULL");
  TuneEntry t;
  if (!cache_lookup(path, key, &t)) return 0;
  *tile_bits = t.tile_bits;
  *split = t.split;
  if (ms) *ms = t.ms;
  return 1;
}

int gvqe_tune_cache_put(const char *path, const char *key, int tile_bits, int split, double ms, const char *sweep) {
  g_err.clear();
  if (!path || !key) return fail(GVQE_EINVAL, "path or key is NULL");
  if (tile_bits < 10 || tile_bits > 13) return fail(GVQE_EINVAL, "tile bits %d outside [10, 13]", tile_bits);
  if (split < SPLIT_AUTO || split > SPLIT_ALWAYS + GVQE_MAX_QUBITS) return fail(GVQE_EINVAL, "split mode %d", split);
  TuneEntry t;
  t.tile_bits = tile_bits;
  t.split = split;
  t.ms = ms;
  t.sweep = sweep ? sweep : "";
  return cache_store(path, key, t);
}

int gvqe_tune_key(gvqe_ansatz a, gvqe_hamiltonian h, int batch, int flags, char *buf, int buflen) {
  g_err.clear();
  if (!a || a->magic != MAGIC_ANSATZ) return fail(GVQE_EINVAL, "invalid ansatz handle");
  if (!h || h->magic != MAGIC_HAM) return fail(GVQE_EINVAL, "invalid Hamiltonian handle");
  if (batch < 1) return fail(GVQE_EINVAL, "batch=%d < 1", batch);
  char name[256] = "no-gpu";
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess)
    snprintf(name, sizeof(name), "%s", prop.name);
  else
    cudaGetLastError();
  const bool cplx = a->gates == 2;
  const bool diag = cplx ? h->cgm.empty() : h->gm.empty();
  char key[512];
  snprintf(key, sizeof(key), "gpu=%s;n=%d;reps=%d;ent=%d;gates=%d;prec=%s;grad=%d;diag=%d;batch=%d", name, a->n,
           a->reps, a->ent, a->gates, (flags & GVQE_FP64) ? "fp64" : "fp32", (flags & GVQE_TUNE_ENERGY) ? 0 : 1,
           diag ? 1 : 0, batch);
  put_report(key, buf, buflen);
  return GVQE_OK;
}

int gvqe_autotune(gvqe_ansatz a, gvqe_hamiltonian h, const double *params, int batch, int flags,
                  const char *cache_path, char *report, int report_len, void *stream) {
  g_err.clear();
  if (!a || a->magic != MAGIC_ANSATZ) return fail(GVQE_EINVAL, "invalid ansatz handle");
  if (!h || h->magic != MAGIC_HAM) return fail(GVQE_EINVAL, "invalid Hamiltonian handle");
  if (a->n != h->n) return fail(GVQE_EINVAL, "ansatz has %d qubits but the Hamiltonian %d", a->n, h->n);
  if (!params) return fail(GVQE_EINVAL, "params is NULL");
  if (batch < 1) return fail(GVQE_EINVAL, "batch=%d < 1", batch);
  if (flags & ~(GVQE_FP64 | GVQE_TUNE_ENERGY)) return fail(GVQE_EINVAL, "unknown flags 0x%x", flags);
  const int prec = flags & GVQE_FP64 ? 1 : 0;
  const bool want_grad = !(flags & GVQE_TUNE_ENERGY);
  cudaStream_t s = (cudaStream_t)stream;
  char keybuf[512];
  int rc = gvqe_tune_key(a, h, batch, flags, keybuf, sizeof(keybuf));
  if (rc != GVQE_OK) return rc;
  const std::string key = keybuf;
  const int tb_max = max_tile_bits(prec);

  if (cache_path && cache_path[0]) {
    TuneEntry t;
    if (cache_lookup(cache_path, key, &t) && t.tile_bits >= 10 && t.tile_bits <= tb_max && t.split >= SPLIT_AUTO &&
        t.split <= SPLIT_ALWAYS + GVQE_MAX_QUBITS) {
      a->tuned_tb[prec] = t.tile_bits;
      a->tuned_split[prec] = t.split;
      a->tuned_xy_tb[prec] = (t.xy_tb >= 10 && t.xy_tb <= tb_max) ? t.xy_tb : 0;
      a->plans.clear();
      char line[256];
      snprintf(line, sizeof(line), "autotune: cached (%s): tile_bits=%d strided=%s%s %.3f ms\n", cache_path,
               t.tile_bits, split_name(t.split).c_str(),
               a->tuned_xy_tb[prec] ? (" xy_tile_bits=" + std::to_string(a->tuned_xy_tb[prec])).c_str() : "", t.ms);
      a->tune_report = std::string(line) + "autotune sweep (cached): " + t.sweep + "\n";
      put_report(a->tune_report, report, report_len);
      return GVQE_OK;
    }
  }

  // candidates: every distinct plan of tile bits 10..max and the two strided layouts
  struct Cand {
    int tb, split;
  };
  std::vector<Cand> cands;
  std::set<std::string> seen;
  // one run per strided pass, or a split first strided pass with y = 1 .. 8 top qubits
  for (int tb = tb_max; tb >= 10; --tb) {
    std::vector<int> modes = {(int)SPLIT_NEVER};
    for (int y = 1; y <= 8; ++y) modes.push_back((int)SPLIT_ALWAYS + y);
    for (int sp : modes) {
      const Plan pl = build_plan(a->n, a->reps, prec, tb, want_grad, true, false, false, a->ent, a->gates, sp);
      std::string d = describe_plan(pl);
      if (seen.insert(d).second) cands.push_back({tb, sp});
    }
  }
  const int P = a->gates * a->n * (a->reps + 1);
  const size_t out_bytes = ((size_t)batch * 8 + 255) / 256 * 256 + (size_t)batch * P * 8;
  rc = a->tune.reserve(out_bytes);
  if (rc != GVQE_OK) return rc;
  double *E = (double *)a->tune.ptr;
  double *G = want_grad ? (double *)((char *)a->tune.ptr + ((size_t)batch * 8 + 255) / 256 * 256) : nullptr;
  EventPair ev;
  GT_CUDA(cudaEventCreate(&ev.a));
  GT_CUDA(cudaEventCreate(&ev.b));
  const int keep_tb = a->tuned_tb[prec], keep_split = a->tuned_split[prec], keep_xy = a->tuned_xy_tb[prec];
  auto restore = [&]() {
    a->tuned_tb[prec] = keep_tb;
    a->tuned_split[prec] = keep_split;
    a->tuned_xy_tb[prec] = keep_xy;
    a->plans.clear();
  };
  // One candidate: a warm-up call (plan, tables, workspaces), then one timed call,
  // two more when a call is short (under 50 ms), averaged.  *per < 0: no memory.
  const int timed = 3;
  auto time_candidate = [&](int tb, int sp, int xtb, double *per) -> int {
    a->tuned_tb[prec] = tb;
    a->tuned_split[prec] = sp;
    a->tuned_xy_tb[prec] = xtb;
    a->plans.clear();
    int r = energy_impl(a, h, params, nullptr, batch, E, G, prec, s);
    if (r == GVQE_ENOMEM) {
      *per = -1.0;
      return GVQE_OK;
    }
    if (r != GVQE_OK) return r;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(GVQE_ECUDA, "autotune candidate tile_bits=%d: %s", tb, cudaGetErrorString(e));
    double total_ms = 0.0;
    int calls = 0;
    while (calls < timed) {
      GT_CUDA(cudaEventRecord(ev.a, s));
      r = energy_impl(a, h, params, nullptr, batch, E, G, prec, s);
      GT_CUDA(cudaEventRecord(ev.b, s));
      GT_CUDA(cudaEventSynchronize(ev.b));
      if (r != GVQE_OK) return r;
      float ms = 0.f;
      GT_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
      total_ms += ms;
      ++calls;
      if (calls == 1 && ms >= 50.f) break;
    }
    *per = total_ms / calls;
    return GVQE_OK;
  };
  std::string sweep;
  // With X/Y strings (RY layers) the X-mask pass's own tile size comes first, on
  // the default plan (its best size hardly depends on the RY passes' layout);
  // the plans are then timed with it.
  const bool cplx = a->gates == 2;
  const bool diag = cplx ? h->cgm.empty() : h->gm.empty();
  int best_xy = 0;
  if (!diag && !cplx) {
    double xy_ms = -1.0;
    for (int xtb = std::min(tb_max, a->n); xtb >= 10; --xtb) {
      double per = 0.0;
      rc = time_candidate(tb_max, SPLIT_AUTO, xtb, &per);
      if (rc != GVQE_OK) {
        restore();
        return rc;
      }
      char line[160];
      snprintf(line, sizeof(line), "%sX-mask tiles 2^%d: %s%.3f ms", sweep.empty() ? "" : "; ", xtb,
               per < 0 ? "no memory " : "", per < 0 ? 0.0 : per);
      sweep += line;
      if (per >= 0 && (xy_ms < 0 || per < xy_ms)) {
        xy_ms = per;
        best_xy = xtb;
      }
    }
  }
  int best = -1;
  double best_ms = 0.0;
  for (size_t c = 0; c < cands.size(); ++c) {
    double per = 0.0;
    rc = time_candidate(cands[c].tb, cands[c].split, best_xy, &per);
    if (rc != GVQE_OK) {
      restore();
      return rc;
    }
    char line[160];
    if (per < 0)
      snprintf(line, sizeof(line), "%stb=%d/%s: no memory", sweep.empty() ? "" : "; ", cands[c].tb,
               split_name(cands[c].split).c_str());
    else
      snprintf(line, sizeof(line), "%stb=%d/%s: %.3f ms", sweep.empty() ? "" : "; ", cands[c].tb,
               split_name(cands[c].split).c_str(), per);
    sweep += line;
    if (per >= 0 && (best < 0 || per < best_ms)) {
      best = (int)c;
      best_ms = per;
    }
  }
  if (best < 0) {
    a->ws.release();
    restore();
    return fail(GVQE_ENOMEM, "autotune: no candidate plan fits in device memory (%s)", sweep.c_str());
  }
  a->ws.release();  // the chosen plan sizes its own workspace on the next call
  a->tuned_tb[prec] = cands[best].tb;
  a->tuned_split[prec] = cands[best].split;
  a->tuned_xy_tb[prec] = best_xy;
  a->plans.clear();
  char line[256];
  snprintf(line, sizeof(line),
           "autotune: measured: tile_bits=%d strided=%s%s %.3f ms per call (batch %d, %s, %s)\n", cands[best].tb,
           split_name(cands[best].split).c_str(),
           best_xy ? (" xy_tile_bits=" + std::to_string(best_xy)).c_str() : "", best_ms, batch,
           want_grad ? "energy+gradient" : "energy", prec ? "fp64" : "fp32");
  a->tune_report = std::string(line) + "autotune sweep: " + sweep + "\n";
  if (cache_path && cache_path[0]) {
    TuneEntry t;
    t.tile_bits = cands[best].tb;
    t.split = cands[best].split;
    t.xy_tb = best_xy;
    t.ms = best_ms;
    t.sweep = sweep;
    rc = cache_store(cache_path, key, t);
    if (rc != GVQE_OK) return rc;
  }
  put_report(a->tune_report, report, report_len);
  return GVQE_OK;
}

}  // extern "C"
