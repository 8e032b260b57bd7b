// Uneven batches: independent bond updates of different bond dimension D and
// gate rank r in one call (the batch variant of the step driver).  Items are
// grouped by kind (D, r); each kind has its own context (plan, tables, work
// space) on its own stream, forked from and joined back into the caller's
// stream by events, so the kinds' pipelines run side by side on the SMs.
// The kinds with the most work per item (the ALS of Fig. 5 grows as K^4 D)
// get the streams of highest priority, so their long pipelines start first
// and the lighter kinds fill the SMs they leave idle.
// The device part of a call -- copies in, every kind's batched update, copies
// out -- can be captured once as one CUDA graph (the fork becomes parallel
// branches) for a given set of per-kind counts and replayed afterwards.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <vector>

#include "../../include/ntu.h"
#include "ntu_impl.h"

namespace {
struct CachedGraph {
  std::vector<int> counts;                // per-kind counts it was captured for
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int launches = 0;                       // kernels in the graph
  void drop() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    counts.clear();
  }
};
}  // namespace

struct ntu_uneven {
  int nk = 0, d = 2, d_anc = 1;
  cudaStream_t stream = nullptr;          // the caller's (or a private) stream
  bool own_stream = false;
  std::vector<cudaStream_t> ks;           // one stream per kind
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  std::vector<ntu_ctx*> ctx;
  std::vector<int> D, r, cap;
  std::vector<size_t> szT;                // complex entries of one site tensor per kind
  std::vector<double2*> h_in, h_out;      // pinned staging per kind: [Ta | Tb | gates], [Ta' | Tb' | info]
  std::vector<int> staged;                // per-kind counts of the inputs on the device
  std::vector<int> order;                 // kinds by decreasing work per item (enqueue order)
  CachedGraph g_host, g_dev;              // copies + update; update only
  int launches = 0;                       // kernels queued by the last run
  char err[256] = {0};
};

namespace {
char g_uneven_err[256] = "no error";

int ufail(ntu_uneven* u, int status, const char* fmt, ...) {
  char* buf = u ? u->err : g_uneven_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, 256, fmt, ap);
  va_end(ap);
  return status;
}

#define UCK(expr, what)                                                        \
  do {                                                                         \
    cudaError_t _e = (expr);                                                   \
    if (_e != cudaSuccess)                                                     \
      return ufail(u, NTU_ECUDA, "%s: %s", what, cudaGetErrorString(_e));      \
  } while (0)

size_t gate_entries(const ntu_uneven* u) { return (size_t)u->d * u->d * u->d * u->d; }

size_t in_entries(const ntu_uneven* u, int k, int n) {
  return (size_t)n * (2 * u->szT[k] + gate_entries(u));
}

// Item bookkeeping of one call: per-kind counts, each item's slot within its
// kind and its offset in the concatenated site-tensor arrays.
struct Layout {
  std::vector<int> cnt, slot;
  std::vector<size_t> off;
};

int layout(ntu_uneven* u, int n, const int* kind, Layout& L) {
  L.cnt.assign(u->nk, 0);
  L.slot.resize(n);
  L.off.resize(n);
  size_t o = 0;
  for (int i = 0; i < n; ++i) {
    const int k = kind[i];
    if (k < 0 || k >= u->nk) return ufail(u, NTU_EINVAL, "item %d: kind %d outside 0..%d", i, k, u->nk - 1);
    if (L.cnt[k] == u->cap[k]) return ufail(u, NTU_EINVAL, "kind %d: more than max_items=%d", k, u->cap[k]);
    L.slot[i] = L.cnt[k]++;
    L.off[i] = o;
    o += u->szT[k];
  }
  return NTU_OK;
}

void pack(ntu_uneven* u, int n, const int* kind, const Layout& L, const double* Ta,
          const double* Tb, const double* gates) {
  const size_t gsz = gate_entries(u);
  const double2 *ta = (const double2*)Ta, *tb = (const double2*)Tb, *gg = (const double2*)gates;
  for (int i = 0; i < n; ++i) {
    const int k = kind[i];
    const size_t st = u->szT[k], nt = (size_t)L.cnt[k] * st;
    double2* hi = u->h_in[k];
    memcpy(hi + (size_t)L.slot[i] * st, ta + L.off[i], st * sizeof(double2));
    memcpy(hi + nt + (size_t)L.slot[i] * st, tb + L.off[i], st * sizeof(double2));
    memcpy(hi + 2 * nt + (size_t)L.slot[i] * gsz, gg + (size_t)i * gsz, gsz * sizeof(double2));
  }
}

void unpack(ntu_uneven* u, int n, const int* kind, const Layout& L, double* Ta_out,
            double* Tb_out, double* info) {
  double2 *oa = (double2*)Ta_out, *ob = (double2*)Tb_out;
  for (int i = 0; i < n; ++i) {
    const int k = kind[i];
    const size_t st = u->szT[k], nt = (size_t)L.cnt[k] * st;
    const double2* ho = u->h_out[k];
    memcpy(oa + L.off[i], ho + (size_t)L.slot[i] * st, st * sizeof(double2));
    memcpy(ob + L.off[i], ho + nt + (size_t)L.slot[i] * st, st * sizeof(double2));
    memcpy(info + (size_t)i * 4, (const double*)(ho + 2 * nt) + (size_t)L.slot[i] * 4,
           4 * sizeof(double));
  }
}

enum : int { PART_IN = 1, PART_UPDATE = 2, PART_OUT = 4 };

// Enqueue the chosen parts for the per-kind counts cnt[] on the kind streams,
// forked from and joined back into the main stream.  per_item: the update of
// every item is its own ntu_batch_update_dev call (the per-bond launch
// sequence); otherwise one batched call per kind.
int enqueue(ntu_uneven* u, const std::vector<int>& cnt, int parts, bool per_item) {
  UCK(cudaEventRecord(u->fork, u->stream), "fork event");
  u->launches = 0;
  for (int kk = 0; kk < u->nk; ++kk) {
    const int k = u->order[kk];
    const int n = cnt[k];
    if (n == 0) continue;
    cudaStream_t s = u->ks[k];
    UCK(cudaStreamWaitEvent(s, u->fork, 0), "fork wait");
    ntu_ctx* c = u->ctx[k];
    ntu::Work& W = c->w;
    const size_t st = u->szT[k], nt = (size_t)n * st;
    const size_t gsz = gate_entries(u), ng = (size_t)n * gsz;
    if (parts & PART_IN) {
      const double2* hi = u->h_in[k];
      UCK(cudaMemcpyAsync(W.Ta_in, hi, nt * sizeof(double2), cudaMemcpyHostToDevice, s), "copy Ta");
      UCK(cudaMemcpyAsync(W.Tb_in, hi + nt, nt * sizeof(double2), cudaMemcpyHostToDevice, s), "copy Tb");
      UCK(cudaMemcpyAsync(W.G_in, hi + 2 * nt, ng * sizeof(double2), cudaMemcpyHostToDevice, s),
          "copy gates");
    }
    if (parts & PART_UPDATE) {
      const int calls = per_item ? n : 1, m = per_item ? 1 : n;
      for (int j = 0; j < calls; ++j) {
        const size_t t0 = (size_t)j * st;
        int e = ntu_batch_update_dev(c, m, (const double*)(W.Ta_in + t0), (const double*)(W.Tb_in + t0),
                                     (const double*)(W.G_in + (size_t)j * gsz),
                                     (double*)(W.Ta_out + t0), (double*)(W.Tb_out + t0),
                                     W.info + (size_t)j * 4);
        if (e) return ufail(u, e, "kind %d: %s", k, ntu_last_error(c));
        u->launches += ntu_last_launch_count(c);
      }
    }
    if (parts & PART_OUT) {
      double2* ho = u->h_out[k];
      UCK(cudaMemcpyAsync(ho, W.Ta_out, nt * sizeof(double2), cudaMemcpyDeviceToHost, s), "copy Ta'");
      UCK(cudaMemcpyAsync(ho + nt, W.Tb_out, nt * sizeof(double2), cudaMemcpyDeviceToHost, s), "copy Tb'");
      UCK(cudaMemcpyAsync(ho + 2 * nt, W.info, (size_t)n * 4 * sizeof(double), cudaMemcpyDeviceToHost, s),
          "copy info");
    }
    UCK(cudaEventRecord(u->join[k], s), "join event");
    UCK(cudaStreamWaitEvent(u->stream, u->join[k], 0), "join wait");
  }
  return NTU_OK;
}

bool any(const std::vector<int>& cnt) {
  for (int c : cnt)
    if (c) return true;
  return false;
}

// Replay (capturing first if the counts changed) the graph of the given parts.
int run_graph(ntu_uneven* u, CachedGraph& G, const std::vector<int>& cnt, int parts) {
  if (!any(cnt)) {
    u->launches = 0;
    return NTU_OK;
  }
  if (!G.exec || G.counts != cnt) {
    G.drop();
    UCK(cudaStreamBeginCapture(u->stream, cudaStreamCaptureModeRelaxed), "begin capture");
    int st = enqueue(u, cnt, parts, false);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(u->stream, &g);
    if (st) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return ufail(u, NTU_ECUDA, "end capture: %s", cudaGetErrorString(e));
    G.graph = g;
    // the kernel nodes keep the priorities of the streams they were captured
    // from (heaviest kinds first), which the replay honours only with this flag
    e = cudaGraphInstantiate(&G.exec, G.graph, cudaGraphInstantiateFlagUseNodePriority);
    if (e != cudaSuccess) {
      G.drop();
      return ufail(u, NTU_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    G.counts = cnt;
    G.launches = u->launches;
  }
  UCK(cudaGraphLaunch(G.exec, u->stream), "graph launch");
  u->launches = G.launches;
  return NTU_OK;
}

int sync_all(ntu_uneven* u, const std::vector<int>& cnt) {
  UCK(cudaStreamSynchronize(u->stream), "stream synchronize");
  for (int k = 0; k < u->nk; ++k) {
    if (cnt[k] == 0) continue;
    int st = ntu_sync(u->ctx[k]);
    if (st) return ufail(u, st, "kind %d: %s", k, ntu_last_error(u->ctx[k]));
  }
  return NTU_OK;
}
}  // namespace

extern "C" const char* ntu_uneven_last_error(const ntu_uneven* u) {
  return u ? u->err : g_uneven_err;
}

extern "C" int ntu_uneven_destroy(ntu_uneven* u) {
  if (!u) return NTU_OK;
  if (u->stream) cudaStreamSynchronize(u->stream);
  u->g_host.drop();
  u->g_dev.drop();
  for (ntu_ctx* c : u->ctx) ntu_destroy(c);
  for (double2* p : u->h_in) if (p) cudaFreeHost(p);
  for (double2* p : u->h_out) if (p) cudaFreeHost(p);
  for (cudaEvent_t e : u->join) if (e) cudaEventDestroy(e);
  if (u->fork) cudaEventDestroy(u->fork);
  for (cudaStream_t s : u->ks) if (s) cudaStreamDestroy(s);
  if (u->own_stream && u->stream) cudaStreamDestroy(u->stream);
  delete u;
  return NTU_OK;
}

extern "C" int ntu_uneven_init(int d_phys, int d_anc, int als_sweeps, int precision, int tau_kmin,
                               int tau_kmax, int n_kinds, const int* D, const int* r,
                               const int* max_items, void* stream, ntu_uneven** out) {
  if (!out || !D || !r || !max_items || n_kinds < 1 || n_kinds > 64)
    return ufail(nullptr, NTU_EINVAL, "ntu_uneven_init: NULL argument or n_kinds outside 1..64");
  *out = nullptr;
  for (int k = 0; k < n_kinds; ++k)
    for (int j = 0; j < k; ++j)
      if (D[j] == D[k] && r[j] == r[k])
        return ufail(nullptr, NTU_EINVAL, "kind %d repeats (D=%d, r=%d)", k, D[k], r[k]);
  ntu_uneven* u = new ntu_uneven();
  u->nk = n_kinds;
  u->d = d_phys;
  u->d_anc = d_anc;
  auto bail = [&](int st, const char* fmt, int k) {
    char keep[256];
    snprintf(keep, sizeof(keep), fmt, k, k < n_kinds ? D[k] : 0, k < n_kinds ? r[k] : 0,
             u->err);
    ntu_uneven_destroy(u);
    memcpy(g_uneven_err, keep, sizeof(keep));
    return st;
  };
  if (stream) {
    u->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&u->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(NTU_ECUDA, "stream creation (kind %d, D=%d, r=%d) %s", 0);
    u->own_stream = true;
  }
  if (cudaEventCreateWithFlags(&u->fork, cudaEventDisableTiming) != cudaSuccess)
    return bail(NTU_ECUDA, "event creation (kind %d, D=%d, r=%d) %s", 0);
  // priority rank of each kind by its per-item work K^4 D (K = D r)
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);   // hi <= lo: numerically lower is higher
  std::vector<int> prio(n_kinds, prio_lo);
  u->order.assign(n_kinds, 0);
  for (int k = 0; k < n_kinds; ++k) {
    const double wk = std::pow((double)D[k] * r[k], 4) * D[k];
    int heavier = 0;                      // rank of kind k by decreasing work, ties by index
    for (int j = 0; j < n_kinds; ++j) {
      const double wj = std::pow((double)D[j] * r[j], 4) * D[j];
      heavier += wj > wk || (wj == wk && j < k);
    }
    prio[k] = prio_hi + heavier < prio_lo ? prio_hi + heavier : prio_lo;
    u->order[heavier] = k;
  }
  for (int k = 0; k < n_kinds; ++k) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, prio[k]) != cudaSuccess)
      return bail(NTU_ECUDA, "stream of kind %d (D=%d, r=%d) %s", k);
    u->ks.push_back(s);
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return bail(NTU_ECUDA, "event of kind %d (D=%d, r=%d) %s", k);
    u->join.push_back(e);
    ntu_config cf;
    memset(&cf, 0, sizeof(cf));
    cf.D = D[k]; cf.d_phys = d_phys; cf.d_anc = d_anc; cf.r = r[k];
    cf.als_sweeps = als_sweeps; cf.precision = precision;
    cf.tau_kmin = tau_kmin; cf.tau_kmax = tau_kmax; cf.max_batch = max_items[k];
    ntu_ctx* c = nullptr;
    // kinds share the GPU, so splitting an item's ALS over several CTAs pays
    // only where it shortens the critical path: the heaviest kind
    int st = ntu::init_context(&cf, s, &c, u->order[0] == k ? 4 : 1);
    if (st != NTU_OK) {
      snprintf(u->err, sizeof(u->err), ": %s", ntu_last_error(nullptr));
      return bail(st, "kind %d (D=%d, r=%d)%s", k);
    }
    u->ctx.push_back(c);
    u->D.push_back(D[k]);
    u->r.push_back(r[k]);
    u->cap.push_back(max_items[k]);
    const size_t dp = (size_t)d_phys * d_anc;
    u->szT.push_back(dp * D[k] * D[k] * D[k] * D[k]);
    double2 *hi = nullptr, *ho = nullptr;
    const size_t outn = (size_t)max_items[k] * 2 * u->szT.back() + (size_t)max_items[k] * 2;
    if (cudaMallocHost(&hi, in_entries(u, k, max_items[k]) * sizeof(double2)) != cudaSuccess ||
        cudaMallocHost(&ho, outn * sizeof(double2)) != cudaSuccess) {
      if (hi) cudaFreeHost(hi);
      return bail(NTU_ENOMEM, "pinned staging of kind %d (D=%d, r=%d) %s", k);
    }
    u->h_in.push_back(hi);
    u->h_out.push_back(ho);
  }
  u->staged.assign(n_kinds, 0);
  *out = u;
  return NTU_OK;
}

extern "C" int ntu_uneven_update_host(ntu_uneven* u, int n, const int* kind, const double* Ta,
                                      const double* Tb, const double* gates, double* Ta_out,
                                      double* Tb_out, double* info, int use_graph) {
  if (!u) return ufail(nullptr, NTU_EINVAL, "NULL uneven context");
  if (n < 0) return ufail(u, NTU_EINVAL, "n=%d", n);
  if (n == 0) return NTU_OK;
  if (!kind || !Ta || !Tb || !gates || !Ta_out || !Tb_out || !info)
    return ufail(u, NTU_EINVAL, "ntu_uneven_update_host: NULL argument");
  Layout L;
  int st = layout(u, n, kind, L);
  if (st) return st;
  pack(u, n, kind, L, Ta, Tb, gates);
  const int parts = PART_IN | PART_UPDATE | PART_OUT;
  st = use_graph ? run_graph(u, u->g_host, L.cnt, parts) : enqueue(u, L.cnt, parts, false);
  if (st) return st;
  st = sync_all(u, L.cnt);
  if (st) return st;
  u->staged = L.cnt;
  unpack(u, n, kind, L, Ta_out, Tb_out, info);
  return NTU_OK;
}

extern "C" int ntu_uneven_stage(ntu_uneven* u, int n, const int* kind, const double* Ta,
                                const double* Tb, const double* gates) {
  if (!u) return ufail(nullptr, NTU_EINVAL, "NULL uneven context");
  if (n < 0) return ufail(u, NTU_EINVAL, "n=%d", n);
  if (n > 0 && (!kind || !Ta || !Tb || !gates))
    return ufail(u, NTU_EINVAL, "ntu_uneven_stage: NULL argument");
  Layout L;
  int st = layout(u, n, kind, L);
  if (st) return st;
  pack(u, n, kind, L, Ta, Tb, gates);
  st = enqueue(u, L.cnt, PART_IN, false);
  if (st) return st;
  st = sync_all(u, L.cnt);
  if (st) return st;
  u->staged = L.cnt;
  return NTU_OK;
}

extern "C" int ntu_uneven_run(ntu_uneven* u, int mode) {
  if (!u) return ufail(nullptr, NTU_EINVAL, "NULL uneven context");
  switch (mode) {
    case NTU_UNEVEN_GROUPED: return enqueue(u, u->staged, PART_UPDATE, false);
    case NTU_UNEVEN_GRAPH: return run_graph(u, u->g_dev, u->staged, PART_UPDATE);
    case NTU_UNEVEN_PER_ITEM: return enqueue(u, u->staged, PART_UPDATE, true);
    default: return ufail(u, NTU_EINVAL, "mode=%d", mode);
  }
}

extern "C" int ntu_uneven_fetch(ntu_uneven* u, int n, const int* kind, double* Ta_out,
                                double* Tb_out, double* info) {
  if (!u) return ufail(nullptr, NTU_EINVAL, "NULL uneven context");
  if (n < 0) return ufail(u, NTU_EINVAL, "n=%d", n);
  if (n > 0 && (!kind || !Ta_out || !Tb_out || !info))
    return ufail(u, NTU_EINVAL, "ntu_uneven_fetch: NULL argument");
  Layout L;
  int st = layout(u, n, kind, L);
  if (st) return st;
  if (L.cnt != u->staged)
    return ufail(u, NTU_ESTATE, "ntu_uneven_fetch: per-kind counts differ from the staged items");
  st = enqueue(u, L.cnt, PART_OUT, false);
  if (st) return st;
  st = sync_all(u, L.cnt);
  if (st) return st;
  unpack(u, n, kind, L, Ta_out, Tb_out, info);
  return NTU_OK;
}

extern "C" int ntu_uneven_sync(ntu_uneven* u) {
  if (!u) return ufail(nullptr, NTU_EINVAL, "NULL uneven context");
  return sync_all(u, u->staged);
}

extern "C" int ntu_uneven_last_launch_count(const ntu_uneven* u) { return u ? u->launches : 0; }

extern "C" int ntu_uneven_set_tuning(ntu_uneven* u, int kind, const ntu_tuning* t) {
  if (!u || !t) return ufail(u, NTU_EINVAL, "ntu_uneven_set_tuning: NULL argument");
  if (kind < 0 || kind >= u->nk) return ufail(u, NTU_EINVAL, "kind %d outside 0..%d", kind, u->nk - 1);
  const int st = ntu_set_tuning(u->ctx[kind], t);
  if (st != NTU_OK)
    return ufail(u, st, "kind %d (D=%d, r=%d): %s", kind, u->D[kind], u->r[kind],
                 ntu_last_error(u->ctx[kind]));
  u->g_host.drop();
  u->g_dev.drop();
  return NTU_OK;
}

extern "C" int ntu_uneven_get_tuning(const ntu_uneven* u, int kind, ntu_tuning* t,
                                     int* split_max) {
  if (!u || !t) return ufail(const_cast<ntu_uneven*>(u), NTU_EINVAL, "ntu_uneven_get_tuning: NULL argument");
  if (kind < 0 || kind >= u->nk)
    return ufail(const_cast<ntu_uneven*>(u), NTU_EINVAL, "kind %d outside 0..%d", kind, u->nk - 1);
  return ntu_get_tuning(u->ctx[kind], t, split_max);
}
