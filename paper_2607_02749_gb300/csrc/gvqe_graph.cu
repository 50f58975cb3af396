// gvqe_graph.cu -- host-side Hamiltonian partitioning (Section IV-C): the
// weighted qubit interaction graph of Eq. 9 and its Louvain partition into
// blocks maximising the modularity of Eq. 10 (with a resolution gamma,
// Section VI-C), followed by the S_min merge of small blocks.
//
// Graphs have at most a few hundred nodes (one per qubit), so every level is a
// dense row-major matrix.  The procedure is deterministic: nodes are visited in
// ascending order, a node moves only when the best gain beats staying by more
// than a relative 1e-12, near-equal gains go to the lowest community label,
// and communities are relabelled by their lowest member after every level.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gvqe.h"
#include "gvqe_internal.h"

namespace gvqe {
namespace {

constexpr double kRelTie = 1e-12;

// Relabel so that labels appear in order of their lowest member; returns the count.
int canonicalise(std::vector<int> &lab) {
  std::vector<int> map(lab.size() + 1, -1);
  int next = 0;
  for (int &c : lab) {
    if (map[c] < 0) map[c] = next++;
    c = map[c];
  }
  return next;
}

// One Louvain level on the dense symmetric matrix a (N x N, self-loops on the
// diagonal after aggregation): returns the community of each node.
std::vector<int> move_nodes(const std::vector<double> &a, int N, double gamma, double two_m) {
  std::vector<double> deg(N, 0.0);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) deg[i] += a[(size_t)i * N + j];
  std::vector<int> comm(N);
  std::vector<double> tot(deg);
  for (int i = 0; i < N; ++i) comm[i] = i;
  std::vector<double> link(N, 0.0);  // weight from the current node to each community
  std::vector<char> seen(N, 0);
  std::vector<int> touched;
  touched.reserve(N);
  bool any = true;
  while (any) {
    any = false;
    for (int i = 0; i < N; ++i) {
      const int from = comm[i];
      tot[from] -= deg[i];
      touched.clear();
      for (int j = 0; j < N; ++j) {
        const double v = a[(size_t)i * N + j];
        if (j == i || v == 0.0) continue;
        const int c = comm[j];
        if (!seen[c]) {
          seen[c] = 1;
          touched.push_back(c);
        }
        link[c] += v;
      }
      auto gain = [&](int c) { return link[c] - gamma * tot[c] * deg[i] / two_m; };
      const double g_stay = gain(from);
      const double tol = kRelTie * std::max(std::max(std::fabs(g_stay), deg[i]), 1e-300);
      double g_top = g_stay;
      for (int c : touched) g_top = std::max(g_top, gain(c));
      int to = from;
      if (g_top > g_stay + tol) {
        to = N;
        for (int c : touched)
          if (gain(c) >= g_top - tol) to = std::min(to, c);
        any = true;
      }
      comm[i] = to;
      tot[to] += deg[i];
      for (int c : touched) {
        link[c] = 0.0;
        seen[c] = 0;
      }
    }
  }
  return comm;
}

std::vector<int> louvain(const std::vector<double> &w, int n, double gamma) {
  double two_m = 0.0;
  for (double v : w) two_m += v;
  std::vector<int> label(n);
  for (int i = 0; i < n; ++i) label[i] = i;
  if (two_m == 0.0) return label;
  std::vector<double> a(w);
  int N = n;
  for (;;) {
    std::vector<int> comm = move_nodes(a, N, gamma, two_m);
    const int nc = canonicalise(comm);
    if (nc == N) break;
    for (int &c : label) c = comm[c];
    std::vector<double> b((size_t)nc * nc, 0.0);
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) b[(size_t)comm[i] * nc + comm[j]] += a[(size_t)i * N + j];
    a.swap(b);
    N = nc;
  }
  canonicalise(label);
  return label;
}

// Merge blocks smaller than s_min: the smallest block (lowest label on ties)
// joins the block it shares the most weight with (lowest label on ties), or,
// sharing none, the smallest other block.
void merge_small(const std::vector<double> &w, int n, int s_min, std::vector<int> &label) {
  for (;;) {
    const int nb = canonicalise(label);
    if (nb <= 1) return;
    std::vector<int> size(nb, 0);
    for (int c : label) size[c] += 1;
    int small = 0;
    for (int b = 1; b < nb; ++b)
      if (size[b] < size[small]) small = b;
    if (size[small] >= s_min) return;
    std::vector<double> shared(nb, 0.0);
    for (int i = 0; i < n; ++i) {
      if (label[i] != small) continue;
      for (int j = 0; j < n; ++j)
        if (label[j] != small) shared[label[j]] += w[(size_t)i * n + j];
    }
    int target = -1;
    for (int b = 0; b < nb; ++b) {
      if (b == small || shared[b] <= 0.0) continue;
      if (target < 0 || shared[b] > shared[target]) target = b;
    }
    if (target < 0) {
      for (int b = 0; b < nb; ++b) {
        if (b == small) continue;
        if (target < 0 || size[b] < size[target]) target = b;
      }
    }
    for (int &c : label)
      if (c == small) c = target;
  }
}

double modularity(const std::vector<double> &w, int n, const std::vector<int> &label, double gamma) {
  double two_m = 0.0;
  std::vector<double> deg(n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      deg[i] += w[(size_t)i * n + j];
      two_m += w[(size_t)i * n + j];
    }
  if (two_m == 0.0) return 0.0;
  double q = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (label[i] == label[j]) q += w[(size_t)i * n + j] - gamma * deg[i] * deg[j] / two_m;
  return q / two_m;
}

}  // namespace
}  // namespace gvqe

using namespace gvqe;

extern "C" {

int gvqe_interaction_graph(int n_qubits, int n_terms, const char *pauli, const double *coeffs, double *w) {
  g_err.clear();
  if (n_qubits < 1 || n_qubits > GVQE_GRAPH_MAX_NODES)
    return fail(GVQE_EINVAL, "n_qubits=%d outside [1, %d]", n_qubits, GVQE_GRAPH_MAX_NODES);
  if (n_terms < 0 || !w || (n_terms > 0 && (!pauli || !coeffs))) return fail(GVQE_EINVAL, "bad arrays");
  const int n = n_qubits;
  std::fill(w, w + (size_t)n * n, 0.0);
  std::vector<int> support;
  for (int k = 0; k < n_terms; ++k) {
    const char *s = pauli + (size_t)k * n;
    support.clear();
    for (int q = 0; q < n; ++q) {
      const char ch = s[q];
      if (ch != 'I' && ch != 'X' && ch != 'Y' && ch != 'Z')
        return fail(GVQE_EINVAL, "term %d: letter '%c' at qubit %d", k, ch, q);
      if (ch != 'I') support.push_back(q);
    }
    if (!std::isfinite(coeffs[k])) return fail(GVQE_EINVAL, "term %d: coefficient not finite", k);
    const double c = std::fabs(coeffs[k]);
    for (int i : support)
      for (int j : support)
        if (i != j) w[(size_t)i * n + j] += c;
  }
  return GVQE_OK;
}

int gvqe_partition(int n, const double *w, double resolution, int min_block, int *block_of, int *n_blocks,
                   double *modularity_out) {
  g_err.clear();
  if (n < 1 || n > GVQE_GRAPH_MAX_NODES) return fail(GVQE_EINVAL, "n=%d outside [1, %d]", n, GVQE_GRAPH_MAX_NODES);
  if (!w || !block_of) return fail(GVQE_EINVAL, "w or block_of is NULL");
  if (!(resolution >= 0.0) || !std::isfinite(resolution)) return fail(GVQE_EINVAL, "resolution %g", resolution);
  if (min_block < 1) return fail(GVQE_EINVAL, "min_block=%d < 1", min_block);
  std::vector<double> g(w, w + (size_t)n * n);
  for (int i = 0; i < n; ++i) {
    if (g[(size_t)i * n + i] != 0.0) return fail(GVQE_EINVAL, "w[%d][%d] != 0 (no self-loops)", i, i);
    for (int j = 0; j < n; ++j) {
      const double v = g[(size_t)i * n + j];
      if (!(v >= 0.0) || !std::isfinite(v)) return fail(GVQE_EINVAL, "w[%d][%d] = %g", i, j, v);
      if (v != g[(size_t)j * n + i]) return fail(GVQE_EINVAL, "w is not symmetric at (%d, %d)", i, j);
    }
  }
  std::vector<int> label = louvain(g, n, resolution);
  merge_small(g, n, min_block, label);
  const int nb = canonicalise(label);
  for (int i = 0; i < n; ++i) block_of[i] = label[i];
  if (n_blocks) *n_blocks = nb;
  if (modularity_out) *modularity_out = modularity(g, n, label, resolution);
  return GVQE_OK;
}

}  // extern "C"
