// Uneven batches: independent bond updates of different bond dimension D and
// gate rank r in one call (the batch variant of the step driver).  Items are
// grouped by kind (D, r); each kind has its own context (plan, tables, work
// space) on one shared stream, and the whole device part of a call -- the
// host-to-device copies of every kind, every kind's batched update and the
// copies back -- is enqueued on that stream, optionally as one CUDA graph
// that is captured on first use for a given set of per-kind counts and
// replayed afterwards.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "../../include/ntu.h"
#include "ntu_impl.h"

struct ntu_uneven {
  int nk = 0, d = 2, d_anc = 1;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<ntu_ctx*> ctx;
  std::vector<int> D, r, cap;
  std::vector<size_t> szT;                // complex entries of one site tensor per kind
  std::vector<double2*> h_in, h_out;      // pinned staging per kind: [Ta | Tb | gates], [Ta' | Tb' | info]
  std::vector<int> graph_counts;          // per-kind counts the cached graph was captured for
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
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

void drop_graph(ntu_uneven* u) {
  if (u->exec) cudaGraphExecDestroy(u->exec);
  if (u->graph) cudaGraphDestroy(u->graph);
  u->exec = nullptr;
  u->graph = nullptr;
  u->graph_counts.clear();
}

size_t in_entries(const ntu_uneven* u, int k, int n) {
  return (size_t)n * (2 * u->szT[k] + (size_t)u->d * u->d * u->d * u->d);
}
}  // namespace

extern "C" const char* ntu_uneven_last_error(const ntu_uneven* u) {
  return u ? u->err : g_uneven_err;
}

extern "C" int ntu_uneven_destroy(ntu_uneven* u) {
  if (!u) return NTU_OK;
  drop_graph(u);
  for (ntu_ctx* c : u->ctx) ntu_destroy(c);
  for (double2* p : u->h_in) if (p) cudaFreeHost(p);
  for (double2* p : u->h_out) if (p) cudaFreeHost(p);
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
  if (stream) {
    u->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&u->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete u;
      return ufail(nullptr, NTU_ECUDA, "stream creation");
    }
    u->own_stream = true;
  }
  for (int k = 0; k < n_kinds; ++k) {
    ntu_config cf;
    memset(&cf, 0, sizeof(cf));
    cf.D = D[k]; cf.d_phys = d_phys; cf.d_anc = d_anc; cf.r = r[k];
    cf.als_sweeps = als_sweeps; cf.precision = precision;
    cf.tau_kmin = tau_kmin; cf.tau_kmax = tau_kmax; cf.max_batch = max_items[k];
    ntu_ctx* c = nullptr;
    int st = ntu_init(&cf, u->stream, &c);
    if (st != NTU_OK) {
      ufail(u, st, "kind %d (D=%d, r=%d): %s", k, D[k], r[k], ntu_last_error(nullptr));
      char keep[256];
      memcpy(keep, u->err, sizeof(keep));
      ntu_uneven_destroy(u);
      memcpy(g_uneven_err, keep, sizeof(keep));
      return st;
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
      ntu_uneven_destroy(u);
      return ufail(nullptr, NTU_ENOMEM, "pinned staging of kind %d", k);
    }
    u->h_in.push_back(hi);
    u->h_out.push_back(ho);
  }
  *out = u;
  return NTU_OK;
}

// Enqueue the device part for the per-kind counts cnt[] (inputs already in
// the pinned staging): copies in, batched updates, copies out.
static int enqueue(ntu_uneven* u, const std::vector<int>& cnt) {
  for (int k = 0; k < u->nk; ++k) {
    const int n = cnt[k];
    if (n == 0) continue;
    ntu_ctx* c = u->ctx[k];
    ntu::Work& W = c->w;
    const size_t nt = (size_t)n * u->szT[k];
    const size_t ng = (size_t)n * u->d * u->d * u->d * u->d;
    const double2* hi = u->h_in[k];
    UCK(cudaMemcpyAsync(W.Ta_in, hi, nt * sizeof(double2), cudaMemcpyHostToDevice, u->stream), "copy Ta");
    UCK(cudaMemcpyAsync(W.Tb_in, hi + nt, nt * sizeof(double2), cudaMemcpyHostToDevice, u->stream), "copy Tb");
    UCK(cudaMemcpyAsync(W.G_in, hi + 2 * nt, ng * sizeof(double2), cudaMemcpyHostToDevice, u->stream),
        "copy gates");
    int st = ntu_batch_update_dev(c, n, (const double*)W.Ta_in, (const double*)W.Tb_in,
                                  (const double*)W.G_in, (double*)W.Ta_out, (double*)W.Tb_out,
                                  W.info);
    if (st) return ufail(u, st, "kind %d: %s", k, ntu_last_error(c));
    double2* ho = u->h_out[k];
    UCK(cudaMemcpyAsync(ho, W.Ta_out, nt * sizeof(double2), cudaMemcpyDeviceToHost, u->stream), "copy Ta'");
    UCK(cudaMemcpyAsync(ho + nt, W.Tb_out, nt * sizeof(double2), cudaMemcpyDeviceToHost, u->stream),
        "copy Tb'");
    UCK(cudaMemcpyAsync(ho + 2 * nt, W.info, (size_t)n * 4 * sizeof(double), cudaMemcpyDeviceToHost,
                        u->stream), "copy info");
  }
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
  // per-kind counts, offsets of every item in the packed arrays
  std::vector<int> cnt(u->nk, 0), slot(n);
  std::vector<size_t> off(n);
  size_t o = 0;
  for (int i = 0; i < n; ++i) {
    const int k = kind[i];
    if (k < 0 || k >= u->nk) return ufail(u, NTU_EINVAL, "item %d: kind %d outside 0..%d", i, k, u->nk - 1);
    if (cnt[k] == u->cap[k]) return ufail(u, NTU_EINVAL, "kind %d: more than max_items=%d", k, u->cap[k]);
    slot[i] = cnt[k]++;
    off[i] = o;
    o += u->szT[k];
  }
  // pack inputs into the pinned staging, item-major inside each kind
  const size_t gsz = (size_t)u->d * u->d * u->d * u->d;
  const double2 *ta = (const double2*)Ta, *tb = (const double2*)Tb, *gg = (const double2*)gates;
  for (int i = 0; i < n; ++i) {
    const int k = kind[i];
    const size_t st = u->szT[k], nt = (size_t)cnt[k] * st;
    double2* hi = u->h_in[k];
    memcpy(hi + (size_t)slot[i] * st, ta + off[i], st * sizeof(double2));
    memcpy(hi + nt + (size_t)slot[i] * st, tb + off[i], st * sizeof(double2));
    memcpy(hi + 2 * nt + (size_t)slot[i] * gsz, gg + (size_t)i * gsz, gsz * sizeof(double2));
  }
  if (use_graph) {
    if (!u->exec || u->graph_counts != cnt) {
      drop_graph(u);
      UCK(cudaStreamBeginCapture(u->stream, cudaStreamCaptureModeRelaxed), "begin capture");
      int st = enqueue(u, cnt);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(u->stream, &g);
      if (st) { if (g) cudaGraphDestroy(g); return st; }
      if (e != cudaSuccess) return ufail(u, NTU_ECUDA, "end capture: %s", cudaGetErrorString(e));
      u->graph = g;
      UCK(cudaGraphInstantiate(&u->exec, u->graph, 0), "graph instantiate");
      u->graph_counts = cnt;
    }
    UCK(cudaGraphLaunch(u->exec, u->stream), "graph launch");
  } else {
    int st = enqueue(u, cnt);
    if (st) return st;
  }
  UCK(cudaStreamSynchronize(u->stream), "stream synchronize");
  for (int k = 0; k < u->nk; ++k) {
    if (cnt[k] == 0) continue;
    int st = ntu_sync(u->ctx[k]);
    if (st) return ufail(u, st, "kind %d: %s", k, ntu_last_error(u->ctx[k]));
  }
  // unpack outputs
  double2 *oa = (double2*)Ta_out, *ob = (double2*)Tb_out;
  for (int i = 0; i < n; ++i) {
    const int k = kind[i];
    const size_t st = u->szT[k], nt = (size_t)cnt[k] * st;
    const double2* ho = u->h_out[k];
    memcpy(oa + off[i], ho + (size_t)slot[i] * st, st * sizeof(double2));
    memcpy(ob + off[i], ho + nt + (size_t)slot[i] * st, st * sizeof(double2));
    memcpy(info + (size_t)i * 4, (const double*)(ho + 2 * nt) + (size_t)slot[i] * 4, 4 * sizeof(double));
  }
  return NTU_OK;
}
