// multidep.cu -- host side of FEA_SCATTER_MULTIDEP: the subdomain plan of
// Sec. 3.2.2, Alg. "multideps".
//
// The paper cuts the elements into subdomains of Chunk_Size elements, stores
// the subdomain graph (subdomains sharing a node are neighbours), and makes
// one task per subdomain with a COMMUTATIVE dependence on every subdomain of
// its neighbour list (itself included) and PRIORITY = the list's length: two
// tasks whose lists meet never run at the same time, in no fixed order, and
// subdomains with more neighbours go first.  The plan built here is that
// graph for the work items of fea_work_items (runs of `chunk` consecutive
// elements of one type), the priority order, and, for each subdomain, a local
// coloring of its elements (greedy, in element order): a CTA runs the
// subdomain's color classes one after the other, so its threads never add
// into one entry at the same time, and the locks keep every other CTA away.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "fea_internal.cuh"

namespace fea {

void free_multidep_plan(fea_mesh* m) {
  MultidepPlan* P = m->mdep;
  if (!P) return;
  cudaFree(P->items);
  cudaFree(P->nb_off);
  cudaFree(P->nb);
  cudaFree(P->order);
  cudaFree(P->cb_off);
  cudaFree(P->cb);
  for (int t = 0; t < kNumTypes; ++t) cudaFree(P->lists[t]);
  cudaFree(P->state);
  delete P;
  m->mdep = nullptr;
}

template <typename T>
static int upload(T** dst, const std::vector<T>& src) {
  FEA_CUDA(cudaMalloc(dst, std::max<size_t>(1, src.size()) * sizeof(T)));
  if (!src.empty()) FEA_CUDA(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return FEA_OK;
}

static int build_plan(fea_mesh* m, int chunk, MultidepPlan* P) {
  P->chunk = chunk;
  // subdomains: the work items, type by type in enum order
  int64_t n_sub = 0;
  for (int t = 0; t < kNumTypes; ++t) {
    const int64_t n = m->group[t].n;
    for (int64_t f = 0; f < n; f += chunk) {
      WorkItem w;
      w.entry = t;
      w.first = (int32_t)f;
      w.count = (int32_t)std::min<int64_t>(chunk, n - f);
      w.pad = 0;
      P->items_h.push_back(w);
      ++n_sub;
    }
  }
  if (n_sub >= INT32_MAX) return fail(FEA_ERR_INDEX_OVERFLOW, "multidep plan: too many subdomains");
  P->n_sub = n_sub;
  // per-type connectivity and original ids on the host
  std::vector<int32_t> conn[kNumTypes], ids[kNumTypes];
  for (int t = 0; t < kNumTypes; ++t) {
    const TypeGroup& g = m->group[t];
    if (!g.n) continue;
    conn[t].resize((size_t)g.n * nodes_of(t));
    FEA_CUDA(cudaMemcpy(conn[t].data(), g.conn, conn[t].size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    ids[t].resize(g.n);
    if (g.ids)
      FEA_CUDA(cudaMemcpy(ids[t].data(), g.ids, g.n * sizeof(int32_t), cudaMemcpyDeviceToHost));
    else
      std::iota(ids[t].begin(), ids[t].end(), 0);
  }
  const int64_t N = m->n_nodes;
  // local coloring and the per-type launch lists: each subdomain's elements
  // grouped by color, element order inside a color
  P->color_h.assign(m->n_elems, -1);
  P->cb_off_h.assign(n_sub + 1, 0);
  std::vector<uint64_t> mask(N, 0);
  std::vector<int32_t> col;
  for (int64_t s = 0; s < n_sub; ++s) {
    const WorkItem& w = P->items_h[s];
    const int t = w.entry, nn = nodes_of(t);
    if (P->lists_h[t].empty()) P->lists_h[t].resize(m->group[t].n);
    col.assign(w.count, 0);
    int ncol = 0;
    for (int i = 0; i < w.count; ++i) {
      const int32_t* en = conn[t].data() + (size_t)(w.first + i) * nn;
      uint64_t used = 0;
      for (int a = 0; a < nn; ++a) used |= mask[en[a]];
      if (used == ~0ull) return fail(FEA_ERR_UNSUPPORTED, "multidep plan: a subdomain needs more than 64 local colors");
      const int c = __builtin_ctzll(~used);
      col[i] = c;
      ncol = std::max(ncol, c + 1);
      for (int a = 0; a < nn; ++a) mask[en[a]] |= 1ull << c;
    }
    for (int i = 0; i < w.count; ++i) {
      const int32_t* en = conn[t].data() + (size_t)(w.first + i) * nn;
      for (int a = 0; a < nn; ++a) mask[en[a]] = 0;
      P->color_h[ids[t][w.first + i]] = col[i];
    }
    // counting sort by color into list positions first .. first + count
    std::vector<int32_t> start(ncol + 1, 0);
    for (int i = 0; i < w.count; ++i) ++start[col[i] + 1];
    for (int c = 0; c < ncol; ++c) start[c + 1] += start[c];
    for (int c = 0; c <= ncol; ++c) P->cb_h.push_back(w.first + start[c]);
    P->cb_off_h[s + 1] = (int64_t)P->cb_h.size();
    for (int i = 0; i < w.count; ++i) P->lists_h[t][w.first + start[col[i]]++] = w.first + i;
    P->max_colors = std::max(P->max_colors, ncol);
  }
  // node -> subdomains holding it
  std::vector<int64_t> ns_off(N + 1, 0);
  std::vector<int32_t> last(N, -1);
  auto for_nodes = [&](int64_t s, auto&& f) {
    const WorkItem& w = P->items_h[s];
    const int nn = nodes_of(w.entry);
    const int32_t* en = conn[w.entry].data() + (size_t)w.first * nn;
    for (int64_t k = 0; k < (int64_t)w.count * nn; ++k) f(en[k]);
  };
  for (int64_t s = 0; s < n_sub; ++s)
    for_nodes(s, [&](int32_t v) {
      if (last[v] != (int32_t)s) {
        last[v] = (int32_t)s;
        ++ns_off[v + 1];
      }
    });
  for (int64_t v = 0; v < N; ++v) ns_off[v + 1] += ns_off[v];
  std::vector<int32_t> ns(ns_off[N]);
  std::vector<int64_t> cur(ns_off.begin(), ns_off.end() - 1);
  std::fill(last.begin(), last.end(), -1);
  for (int64_t s = 0; s < n_sub; ++s)
    for_nodes(s, [&](int32_t v) {
      if (last[v] != (int32_t)s) {
        last[v] = (int32_t)s;
        ns[cur[v]++] = (int32_t)s;
      }
    });
  // neighbour lists (ascending: the order locks are taken in)
  P->nb_off_h.assign(n_sub + 1, 0);
  std::vector<int32_t> stamp(n_sub, -1), lst;
  for (int64_t s = 0; s < n_sub; ++s) {
    lst.clear();
    for_nodes(s, [&](int32_t v) {
      for (int64_t k = ns_off[v]; k < ns_off[v + 1]; ++k)
        if (stamp[ns[k]] != (int32_t)s) {
          stamp[ns[k]] = (int32_t)s;
          lst.push_back(ns[k]);
        }
    });
    std::sort(lst.begin(), lst.end());
    P->nb_h.insert(P->nb_h.end(), lst.begin(), lst.end());
    P->nb_off_h[s + 1] = (int64_t)P->nb_h.size();
    P->max_nb = std::max<int64_t>(P->max_nb, (int64_t)lst.size());
  }
  // priority: more neighbours first (the paper's PRIORITY(nneig)); ties in a
  // hashed order, which spreads subdomains of equal priority over the mesh
  // (in id order, neighbours follow one another and block each other)
  auto tie = [](uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
  };
  P->order_h.resize(n_sub);
  std::iota(P->order_h.begin(), P->order_h.end(), 0);
  std::sort(P->order_h.begin(), P->order_h.end(), [&](int32_t a, int32_t b) {
    const int64_t da = P->nb_off_h[a + 1] - P->nb_off_h[a], db = P->nb_off_h[b + 1] - P->nb_off_h[b];
    if (da != db) return da > db;
    const uint32_t ha = tie((uint32_t)a), hb = tie((uint32_t)b);
    return ha != hb ? ha < hb : a < b;
  });
  // device copies; state, locks and the two control words in one array
  int rc = upload(&P->items, P->items_h);
  if (!rc) rc = upload(&P->nb_off, P->nb_off_h);
  if (!rc) rc = upload(&P->nb, P->nb_h);
  if (!rc) rc = upload(&P->order, P->order_h);
  if (!rc) rc = upload(&P->cb_off, P->cb_off_h);
  if (!rc) rc = upload(&P->cb, P->cb_h);
  for (int t = 0; t < kNumTypes && !rc; ++t)
    if (!P->lists_h[t].empty()) rc = upload(&P->lists[t], P->lists_h[t]);
  if (rc) return rc;
  FEA_CUDA(cudaMalloc(&P->state, (2 * n_sub + 2) * sizeof(int32_t)));
  P->locks = P->state + n_sub;
  P->ctrl = P->locks + n_sub;
  return FEA_OK;
}

int ensure_multidep_plan(fea_mesh* m, int chunk, MultidepPlan** out) {
  if (chunk <= 0 || chunk > (1 << 24)) return fail(FEA_ERR_ARG, "multidep: chunk must be in [1, 2^24]");
  if (m->mdep && m->mdep->chunk == chunk) {
    *out = m->mdep;
    return FEA_OK;
  }
  free_multidep_plan(m);
  MultidepPlan* P = new MultidepPlan();
  int rc = build_plan(m, chunk, P);
  if (rc) {
    m->mdep = P;  // freed through the mesh's own release path
    free_multidep_plan(m);
    return rc;
  }
  m->mdep = P;
  *out = P;
  return FEA_OK;
}

// per-launch reset: every subdomain pending, every lock free (but the one a
// test holds), hint and done count zero
int reset_multidep(const MultidepPlan& P, cudaStream_t s) {
  FEA_CUDA(cudaMemsetAsync(P.state, 0, (2 * P.n_sub + 2) * sizeof(int32_t), s));
  if (P.held >= 0) FEA_CUDA(cudaMemsetAsync(P.locks + P.held, 1, sizeof(int32_t), s));
  return FEA_OK;
}

}  // namespace fea

using namespace fea;

extern "C" int fea_multidep_plan(fea_mesh* m, int chunk, int64_t info[4], int64_t* nb_off_h, int32_t* nb_h,
                                 int32_t* order_h, int32_t* color_h) {
  if (!m || !info) return fail(FEA_ERR_ARG, "fea_multidep_plan: null argument");
  if (chunk < 0) return fail(FEA_ERR_ARG, "fea_multidep_plan: chunk must be >= 0");
  MultidepPlan* P = nullptr;
  int rc = ensure_multidep_plan(m, chunk ? chunk : 128, &P);
  if (rc) return rc;
  info[0] = P->n_sub;
  info[1] = (int64_t)P->nb_h.size();
  info[2] = P->max_nb;
  info[3] = P->max_colors;
  if (nb_off_h) std::memcpy(nb_off_h, P->nb_off_h.data(), P->nb_off_h.size() * sizeof(int64_t));
  if (nb_h) std::memcpy(nb_h, P->nb_h.data(), P->nb_h.size() * sizeof(int32_t));
  if (order_h) std::memcpy(order_h, P->order_h.data(), P->order_h.size() * sizeof(int32_t));
  if (color_h) std::memcpy(color_h, P->color_h.data(), P->color_h.size() * sizeof(int32_t));
  return FEA_OK;
}

extern "C" int fea_multidep_hold(fea_mesh* m, int subdomain, int held) {
  if (!m || !m->mdep) return fail(FEA_ERR_ARG, "fea_multidep_hold: no multidep plan on this mesh");
  if (subdomain < 0 || subdomain >= m->mdep->n_sub)
    return fail(FEA_ERR_ARG, "fea_multidep_hold: subdomain out of range");
  if (held)
    m->mdep->held = subdomain;
  else if (m->mdep->held == subdomain)
    m->mdep->held = -1;
  return FEA_OK;
}
