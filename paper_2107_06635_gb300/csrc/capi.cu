// C ABI of the NTU library (include/ntu.h): context and work-space
// management, argument validation, and the host-side sequencing of the
// kernels of one bond update.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "ntu_dev.cuh"
#include "ntu_impl.h"

using namespace ntu;

// Errors of calls without a context (ntu_init, ntu_gate_qr_noalloc): one
// message per host thread, read by ntu_last_error(NULL) on that thread.
static thread_local char g_noctx_err[320] = "";

int ntu::fail(ntu_ctx* c, int status, const char* fmt, ...) {
  char* buf = c ? c->err : g_noctx_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, 320, fmt, ap);
  va_end(ap);
  return status;
}

cudaError_t ntu::after_launch(ntu_ctx* c, const char* name) {
  c->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && c->debug_sync) {
    e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e != cudaSuccess && c->debug_sync)
    fprintf(stderr, "ntu: kernel %s failed: %s\n", name, cudaGetErrorString(e));
  if (e == cudaSuccess && c->debug_sync) {
    int st[2] = {0, 0};
    if (cudaMemcpy(st, c->d_status, sizeof(st), cudaMemcpyDeviceToHost) == cudaSuccess && st[0])
      fprintf(stderr, "ntu: status %d (reason 0x%x) set by or before kernel %s (launch %d)\n",
              st[0], st[1], name, c->launches);
  }
  return e;
}

static int cuda_check(ntu_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return NTU_OK;
  int st = (e == cudaErrorMemoryAllocation) ? NTU_ENOMEM : NTU_ECUDA;
  return fail(c, st, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(expr, what)                                   \
  do {                                                   \
    int _s = cuda_check(c, (expr), what);                \
    if (_s != NTU_OK) return _s;                         \
  } while (0)

// --------------------------------------------------------- work space
namespace {
struct Carver {
  char* base = nullptr;
  size_t off = 0;
  bool dry = true;
  template <typename T> T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~(size_t)255;
    T* p = dry ? nullptr : reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};

void carve(ntu_ctx* c, Carver& cv) {
  Plan& P = c->plan;
  Work& W = c->w;
  const size_t n = W.cap;
  const size_t es = c->env_es;
  const size_t d2r = (size_t)P.d * P.d * P.r, mK = (size_t)P.m * P.K;
  W.GA = cv.take<double2>(n * d2r);
  W.GB = cv.take<double2>(n * d2r);
  W.Mg = cv.take<double2>(n * 2 * mK);
  W.Qcm = cv.take<double2>(n * 2 * mK);
  W.QA = cv.take<double2>(n * mK);
  W.QB = cv.take<double2>(n * mK);
  W.RA = cv.take<double2>(n * P.szR);
  W.RB = cv.take<double2>(n * P.szR);
  bool mixed = c->cfg.precision != NTU_FP64;
  W.Tac = mixed ? (void*)cv.take<char>(n * P.szT * es) : nullptr;
  W.Tbc = mixed ? (void*)cv.take<char>(n * P.szT * es) : nullptr;
  W.QAc = mixed ? (void*)cv.take<char>(n * P.szQ * es) : nullptr;
  W.QBc = mixed ? (void*)cv.take<char>(n * P.szQ * es) : nullptr;
  const bool tc = c->cfg.precision == NTU_MIXED_BF16X3;
  W.EL = cv.take<char>(n * P.szE1 * es);
  W.ER = cv.take<char>(n * P.szE1 * es);
  W.Y = cv.take<char>(n * P.szQ * es);
  if (!tc) {
    W.ETL = cv.take<char>(n * P.szE2 * es);
    W.EBL = cv.take<char>(n * P.szE2 * es);
    W.ETR = cv.take<char>(n * P.szE2 * es);
    W.EBR = cv.take<char>(n * P.szE2 * es);
    W.T1 = cv.take<char>(n * P.szS2 * es);
    W.T2 = cv.take<char>(n * P.szS2 * es);
    W.HL = cv.take<char>(n * P.szS2 * es);
    W.HR = cv.take<char>(n * P.szS2 * es);
  } else {
    // split BF16 operands (2 bytes each, rows x [hi | lo])
    const size_t bE = (size_t)P.rowsE * 2 * P.krpE * 2, bT = (size_t)P.rowsT * 2 * P.krpE * 2;
    W.ETLd = cv.take<char>(n * bE);
    W.EBLd = cv.take<char>(n * bE);
    W.ETRd = cv.take<char>(n * bE);
    W.EBRd = cv.take<char>(n * bE);
    W.T2s = cv.take<char>(n * bT);
    W.HLd = cv.take<char>(n * (size_t)P.rowsHL * 2 * P.krpJ * 2);
    W.HRs = cv.take<char>(n * (size_t)P.rowsHR * 2 * P.krpJ * 2);
    W.Ys = cv.take<char>(n * (size_t)P.rowsY * 2 * P.krpY * 2);
    W.Qs = cv.take<char>(n * (size_t)P.rowsQ * 2 * P.krpY * 2);
  }
  W.qrflag = cv.take<int>(n * 2);
  W.graw = cv.take<double2>(n * P.szG);
  W.g = cv.take<double2>(n * P.szG);
  W.gscr = cv.take<double2>(n * P.szG);
  W.gw = cv.take<double2>(n * P.szG);
  W.gz = cv.take<double>(n * P.szG);
  W.geig = cv.take<double>(n * 2 * P.ng);
  W.gtau = cv.take<double2>(n * P.ng);
  W.gp = cv.take<double2>(n * P.ng);
  W.diag = cv.take<double>(n * 3);
  // ALS scratch private to each CTA: an item's ALS may run on als_split CTAs
  const size_t na = n * (size_t)W.als_split;
  W.x0 = cv.take<double2>(na * P.ng);
  W.gx0 = cv.take<double2>(na * P.ng);
  W.Tm = cv.take<double2>(na * (size_t)P.ng * P.nA);
  W.gA = cv.take<double2>(na * (size_t)P.nA * P.nA);
  W.gC = cv.take<double2>(na * (size_t)P.nA * P.nA);
  W.jv = cv.take<double2>(na * P.nA);
  W.pv = cv.take<double2>(na * P.nA);
  W.tauv = cv.take<double2>(na * P.nA);
  W.dv = cv.take<double>(na * P.nA);
  W.ev = cv.take<double>(na * P.nA);
  W.rotcap = 6 * P.nA * P.nA + 64;
  W.rc = cv.take<double>(na * W.rotcap);
  W.rs = cv.take<double>(na * W.rotcap);
  W.rk = cv.take<int>(na * W.rotcap);
  W.als_sync = cv.take<int>(n);
  W.gmaxb = cv.take<unsigned long long>(n);
  W.gscale = cv.take<int>(n);
  W.MA = cv.take<double2>(n * (size_t)P.K * P.D);
  W.MB = cv.take<double2>(n * (size_t)P.K * P.D);
  W.info = cv.take<double>(n * 4 + 16);
  W.Ta_out = cv.take<double2>(n * P.szT);
  W.Tb_out = cv.take<double2>(n * P.szT);
  W.Ta_in = cv.take<double2>(n * P.szT);
  W.Tb_in = cv.take<double2>(n * P.szT);
  const size_t d4 = (size_t)P.d * P.d * P.d * P.d;
  W.G_in = cv.take<double2>(n * d4);
  W.A = cv.take<double2>(P.szT);
  W.B = cv.take<double2>(P.szT);
  W.cTa = cv.take<double2>(P.szT);
  W.cTb = cv.take<double2>(P.szT);
  W.cA2 = cv.take<double2>(P.szT);
  W.cB2 = cv.take<double2>(P.szT);
  W.cG = cv.take<double2>(4 * d4);
  W.op = cv.take<double2>(2 * (size_t)P.d * P.d);
  W.mscr1 = cv.take<double2>(P.szT);
  W.mscr2 = cv.take<double2>(P.szT);
  W.medge = cv.take<double2>(4 * (size_t)P.D * P.D);
  W.mval = cv.take<double2>(2);
  W.lam = cv.take<double>(4 * (size_t)P.D);
  // slices of g for the tensor-core ALS build (mixed contexts, K = 16 or
  // 32): both ALS steps' box rows of 128 bytes, 3 MB (K = 16) or 48 MB
  // (K = 32) per item, left out beyond 24 GB in all
  const size_t oz_item = (size_t)2 * oz_rows_side(P.K) * 128;
  const bool oz = mixed && oz_item > 0 && n * oz_item <= ((size_t)24 << 30);
  W.gsl = oz ? (void*)cv.take<char>(n * oz_item) : nullptr;
  W.gexp = oz ? cv.take<short>(n * (size_t)2 * P.K * P.ng) : nullptr;
  W.gmap = oz ? cv.take<CUtensorMap>(1) : nullptr;
}
}  // namespace

static int check_status(ntu_ctx* c) {
  int st[2] = {0, 0};
  CK(cudaStreamSynchronize(c->stream), "stream synchronize");
  CK(cudaMemcpy(st, c->d_status, sizeof(st), cudaMemcpyDeviceToHost), "read status");
  if (st[0] != 0) {
    int zero[2] = {0, 0};
    cudaMemcpy(c->d_status, zero, sizeof(zero), cudaMemcpyHostToDevice);
    return fail(c, st[0], "device raised status %d (%s; reason bits 0x%x: 1 SVD non-finite, "
                "2 ALS eigen-solver, 4 ALS non-finite error, 8 repair eigen-solver, "
                "16 metric trace not positive, 32 tensor-core wait, 64 ALS exchange "
                "between the CTAs of an item)", st[0],
                st[0] == NTU_ENUMERIC ? "non-finite value or solver non-convergence"
                                      : "bounded wait ran out", st[1]);
  }
  return NTU_OK;
}

// ------------------------------------------------------------- lifecycle
extern "C" int ntu_init(const ntu_config* cfg, void* stream, ntu_ctx** out) {
  return ntu::init_context(cfg, stream, out, 4);
}

// ntu_init with a cap on the number of CTAs one item's ALS may use (the
// uneven-batch driver lets only its heaviest kind split).
int ntu::init_context(const ntu_config* cfg, void* stream, ntu_ctx** out, int max_split) {
  if (!cfg || !out) return fail(nullptr, NTU_EINVAL, "ntu_init: NULL argument");
  *out = nullptr;
  const ntu_config& f = *cfg;
  if (f.D < 1 || f.D > 8) return fail(nullptr, NTU_EINVAL, "D=%d outside 1..8", f.D);
  if (f.d_phys < 2 || f.d_phys > 4) return fail(nullptr, NTU_EINVAL, "d_phys=%d outside 2..4", f.d_phys);
  if (f.d_anc < 1 || f.d_anc > 4) return fail(nullptr, NTU_EINVAL, "d_anc=%d outside 1..4", f.d_anc);
  if (f.r < 1 || f.r > f.d_phys * f.d_phys) return fail(nullptr, NTU_EINVAL, "r=%d outside 1..d^2", f.r);
  if (f.D * f.r > 32) return fail(nullptr, NTU_EINVAL, "D*r=%d exceeds 32", f.D * f.r);
  if (f.d_phys * f.d_anc * f.D * f.D < f.r)
    return fail(nullptr, NTU_EINVAL, "d_p*D^2 < r: gated matrix has fewer rows than columns");
  if (f.als_sweeps < 0 || f.als_sweeps > 1000) return fail(nullptr, NTU_EINVAL, "als_sweeps=%d", f.als_sweeps);
  if (f.precision < 0 || f.precision > 2) return fail(nullptr, NTU_EINVAL, "precision=%d", f.precision);
  if (f.tau_kmin < 0 || f.tau_kmax > 20 || f.tau_kmin > f.tau_kmax)
    return fail(nullptr, NTU_EINVAL, "tau_kmin=%d tau_kmax=%d", f.tau_kmin, f.tau_kmax);
  if (f.max_batch < 1 || f.max_batch > 65535) return fail(nullptr, NTU_EINVAL, "max_batch=%d", f.max_batch);
  if (f.wait_budget < 0) return fail(nullptr, NTU_EINVAL, "wait_budget=%d", f.wait_budget);
  // the fused t1-t2 of the split-BF16 environment holds one 64-wide K tile
  // of Y and conj(Q): 2 d_p D real columns at most
  if (f.precision == NTU_MIXED_BF16X3 && 2 * f.d_phys * f.d_anc * f.D > 64)
    return fail(nullptr, NTU_EUNSUPPORTED,
                "NTU_MIXED_BF16X3 needs 2*d_phys*d_anc*D <= 64 (got %d); use NTU_MIXED_FP32",
                2 * f.d_phys * f.d_anc * f.D);
  ntu_ctx* c = new (std::nothrow) ntu_ctx();
  if (!c) return fail(nullptr, NTU_ENOMEM, "host allocation");
  memset(c, 0, sizeof(*c));
  c->cfg = f;
  c->tune.t12_pair = -1;
  c->use_graphs = 1;
  c->wait_polls = f.wait_budget > 0 ? (long long)f.wait_budget : (1ll << 23);
  c->env_es = f.precision == NTU_FP64 ? sizeof(double2) : sizeof(float2);
  if (stream) { c->stream = (cudaStream_t)stream; c->own_stream = false; }
  else {
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { int st = cuda_check(nullptr, e, "stream"); delete c; return st; }
    c->own_stream = true;
  }
  {
    // the device this context runs on: its SM count sizes the persistent
    // grids, and the kernels' shared-memory limits are set on it
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && c->sms < 1) c->sms = 1;
    if (e == cudaSuccess) e = gate_qr_attributes();
    if (e == cudaSuccess) e = t12_attributes();
    if (e == cudaSuccess) e = tc_attributes();
    if (e != cudaSuccess) {
      int st = cuda_check(nullptr, e, "device attributes");
      if (c->own_stream) cudaStreamDestroy(c->stream);
      delete c;
      return st;
    }
  }
  int st = plan_build(c);
  if (st != NTU_OK) { ntu_destroy(c); return fail(nullptr, st, "plan tables"); }
  c->w.cap = f.max_batch;
  // Batches too small to fill the GPU at three ALS CTAs per SM let each
  // item's ALS run on 2 or 4 CTAs (mixed contexts, whose reduced-metric
  // build is split between them; see k_als).
  c->w.als_split = 1;
  if (f.precision != NTU_FP64) {
    const int room = 3 * c->sms / f.max_batch;
    c->w.als_split = room >= 4 ? 4 : (room >= 2 ? 2 : 1);
    while (c->w.als_split > max_split && c->w.als_split > 1) c->w.als_split >>= 1;
  }
  Carver dry;
  carve(c, dry);
  void* base = nullptr;
  cudaError_t e = cudaMalloc(&base, dry.off);
  if (e != cudaSuccess) {
    ntu_destroy(c);
    return fail(nullptr, NTU_ENOMEM, "device work space of %zu bytes: %s", dry.off,
                cudaGetErrorString(e));
  }
  Carver real;
  real.base = (char*)base;
  real.dry = false;
  carve(c, real);
  // carve() filled every pointer; W.GA is the first slice, i.e. the block base
  e = cudaMalloc(&c->d_status, sizeof(int) * 16);
  if (e != cudaSuccess) { cudaFree(base); ntu_destroy(c); return fail(nullptr, NTU_ENOMEM, "status word"); }
  cudaMemset(c->d_status, 0, sizeof(int) * 16);
  c->d_paths = c->d_status + 8;
  const char* dbg = getenv("NTU_DEBUG_SYNC");
  c->debug_sync = (dbg && dbg[0] == '1') ? 1 : 0;
  cudaMemset(base, 0, dry.off);
  {
    double ones[32];
    for (int i = 0; i < 32; ++i) ones[i] = 1.0;
    cudaMemcpy(c->w.lam, ones, 4 * sizeof(double) * f.D, cudaMemcpyHostToDevice);
  }
  if (f.precision == NTU_MIXED_BF16X3) {
    int prop = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&prop, cudaDevAttrComputeCapabilityMajor, dev);
    if (prop != 10) {
      ntu_destroy(c);
      return fail(nullptr, NTU_EUNSUPPORTED,
                  "NTU_MIXED_BF16X3 needs a compute capability 10.x GPU (tcgen05)");
    }
    st = tc_plan_maps(c);
    if (st != NTU_OK) {
      ntu_destroy(c);
      return fail(nullptr, st, "tensor maps of the split operands");
    }
  }
  if (c->w.gsl) {
    // the tensor-core ALS build needs tcgen05 (compute capability 10.x)
    int major = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    if (major == 10 &&
        tc_make_map(&c->plan.mapGsl, c->w.gsl, 64, 2 * oz_rows_side(c->plan.K), f.max_batch,
                    128) == NTU_OK &&
        cudaMemcpy(c->w.gmap, &c->plan.mapGsl, sizeof(CUtensorMap), cudaMemcpyHostToDevice) ==
            cudaSuccess)
      c->plan.oz_ok = 1;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    ntu_destroy(c);
    return fail(nullptr, NTU_ECUDA, "device synchronize after allocation");
  }
  *out = c;
  return NTU_OK;
}

void ntu::drop_step_graphs(ntu_ctx* c) {
  for (int i = 0; i < 4; ++i) {
    if (c->step_graph[i]) cudaGraphExecDestroy(c->step_graph[i]);
    c->step_graph[i] = nullptr;
  }
}

extern "C" int ntu_destroy(ntu_ctx* c) {
  if (!c) return NTU_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_step_graphs(c);
  if (c->w.GA) cudaFree(c->w.GA);
  if (c->d_status) cudaFree(c->d_status);
  for (int i = 0; i < 6; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamDestroy(c->copy_stream);
  }
  for (int i = 0; i < 3; ++i)
    if (c->cev[i]) cudaEventDestroy(c->cev[i]);
  plan_free(c);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return NTU_OK;
}

extern "C" const char* ntu_last_error(const ntu_ctx* c) { return c ? c->err : g_noctx_err; }

extern "C" int ntu_sync(ntu_ctx* c) {
  if (!c) return fail(nullptr, NTU_EINVAL, "NULL context");
  return check_status(c);
}

extern "C" int ntu_last_launch_count(const ntu_ctx* c) { return c ? c->launches : 0; }

extern "C" int ntu_set_tuning(ntu_ctx* c, const ntu_tuning* t) {
  if (!c || !t) return fail(c, NTU_EINVAL, "ntu_set_tuning: NULL argument");
  if (t->t12_pair < -1 || t->t12_pair > 1)
    return fail(c, NTU_EINVAL, "t12_pair=%d outside -1..1", t->t12_pair);
  if (t->t12_pair == 1 && (c->cfg.D != 8 || c->cfg.precision != NTU_MIXED_BF16X3))
    return fail(c, NTU_EINVAL, "t12_pair=1 needs D=8 on a split-BF16 context");
  if (t->als_ctas_per_sm != 0 && t->als_ctas_per_sm != 2 && t->als_ctas_per_sm != 3)
    return fail(c, NTU_EINVAL, "als_ctas_per_sm=%d: 0, 2 or 3", t->als_ctas_per_sm);
  if (t->als_split != 0 && t->als_split != 1 && t->als_split != 2 && t->als_split != 4)
    return fail(c, NTU_EINVAL, "als_split=%d: 0, 1, 2 or 4", t->als_split);
  if (t->als_split > c->w.als_split)
    return fail(c, NTU_EINVAL, "als_split=%d exceeds the %d this context allocated for",
                t->als_split, c->w.als_split);
  if (t->als_build < 0 || t->als_build > 2)
    return fail(c, NTU_EINVAL, "als_build=%d outside 0..2", t->als_build);
  if (t->als_build == 2 && !c->plan.oz_ok)
    return fail(c, NTU_EINVAL, "als_build=2 needs a mixed context with K = D r = 16 or 32 on "
                "a compute capability 10.x GPU");
  c->tune = *t;
  drop_step_graphs(c);
  return NTU_OK;
}

extern "C" int ntu_get_tuning(const ntu_ctx* c, ntu_tuning* t, int* split_max) {
  if (!c || !t) return fail(const_cast<ntu_ctx*>(c), NTU_EINVAL, "ntu_get_tuning: NULL argument");
  *t = c->tune;
  if (split_max) *split_max = c->w.als_split;
  return NTU_OK;
}

extern "C" int ntu_set_graphs(ntu_ctx* c, int on) {
  if (!c) return fail(c, NTU_EINVAL, "NULL context");
  c->use_graphs = on ? 1 : 0;
  if (!on) drop_step_graphs(c);
  return NTU_OK;
}

extern "C" int ntu_inject_wait_timeout(ntu_ctx* c, int on) {
  if (!c) return fail(c, NTU_EINVAL, "NULL context");
  if (c->w.als_split < 2)
    return fail(c, NTU_EUNSUPPORTED, "this context's ALS runs one CTA per item: no rendezvous");
  c->inject_timeout = on ? 1 : 0;
  drop_step_graphs(c);
  return NTU_OK;
}

extern "C" int ntu_solver_paths(ntu_ctx* c, int* counts) {
  if (!c || !counts) return fail(c, NTU_EINVAL, "ntu_solver_paths: NULL argument");
  CK(cudaStreamSynchronize(c->stream), "stream synchronize");
  CK(cudaMemcpy(counts, c->d_paths, 8 * sizeof(int), cudaMemcpyDeviceToHost), "read counters");
  CK(cudaMemset(c->d_paths, 0, 8 * sizeof(int)), "reset counters");
  return NTU_OK;
}

// ------------------------------------------------------------ unit cell
extern "C" int ntu_set_state(ntu_ctx* c, const double* A, const double* B) {
  if (!c || !A || !B) return fail(c, NTU_EINVAL, "ntu_set_state: NULL argument");
  size_t bytes = c->plan.szT * sizeof(double2);
  CK(cudaMemcpyAsync(c->w.A, A, bytes, cudaMemcpyHostToDevice, c->stream), "copy A");
  CK(cudaMemcpyAsync(c->w.B, B, bytes, cudaMemcpyHostToDevice, c->stream), "copy B");
  c->stage = 0;
  return check_status(c);
}

extern "C" int ntu_get_state(ntu_ctx* c, double* A, double* B) {
  if (!c || !A || !B) return fail(c, NTU_EINVAL, "ntu_get_state: NULL argument");
  size_t bytes = c->plan.szT * sizeof(double2);
  CK(cudaMemcpyAsync(A, c->w.A, bytes, cudaMemcpyDeviceToHost, c->stream), "copy A");
  CK(cudaMemcpyAsync(B, c->w.B, bytes, cudaMemcpyDeviceToHost, c->stream), "copy B");
  return check_status(c);
}

static int cell_gate_qr(ntu_ctx* c, int bond, const double2* gate_dev) {
  Work& W = c->w;
  CK(launch_orient(c, bond, W.A, W.B, W.cTa, W.cTb), "orient");
  CK(launch_gate_qr(c, 1, W.cTa, W.cTb, gate_dev, bond >= 2 ? 1 : 0, W.QA, W.RA, W.QB, W.RB),
     "gate + QR");
  return NTU_OK;
}

static int cell_env(ntu_ctx* c) {
  Work& W = c->w;
  CK(launch_env(c, 1, W.cTa, W.cTb, W.QA, W.QB, W.graw), "environment");
  CK(launch_repair(c, 1, W.graw, c->cfg.precision != NTU_FP64, W.g, W.diag), "repair");
  return NTU_OK;
}

static int cell_als(ntu_ctx* c, int bond, double* info_dev) {
  Work& W = c->w;
  CK(launch_als(c, 1, W.g, W.RA, W.RB, W.MA, W.MB, info_dev), "ALS");
  CK(launch_recompose(c, 1, W.QA, W.QB, W.MA, W.MB, W.cA2, W.cB2), "recompose");
  CK(launch_deorient(c, bond, W.cA2, W.cB2, W.A, W.B), "write back");
  return NTU_OK;
}

extern "C" int ntu_apply_gate(ntu_ctx* c, int bond, const double* gate, double* RA_out,
                              double* RB_out) {
  if (!c || !gate) return fail(c, NTU_EINVAL, "ntu_apply_gate: NULL argument");
  if (bond < 0 || bond > 3) return fail(c, NTU_EINVAL, "bond=%d outside 0..3", bond);
  const Plan& P = c->plan;
  size_t d4 = (size_t)P.d * P.d * P.d * P.d;
  CK(cudaMemcpyAsync(c->w.cG, gate, d4 * sizeof(double2), cudaMemcpyHostToDevice, c->stream),
     "copy gate");
  int st = cell_gate_qr(c, bond, c->w.cG);
  if (st) return st;
  size_t rb = P.szR * sizeof(double2);
  if (RA_out) CK(cudaMemcpyAsync(RA_out, c->w.RA, rb, cudaMemcpyDeviceToHost, c->stream), "copy RA");
  if (RB_out) CK(cudaMemcpyAsync(RB_out, c->w.RB, rb, cudaMemcpyDeviceToHost, c->stream), "copy RB");
  st = check_status(c);
  if (st) return st;
  c->stage = 1;
  c->stage_bond = bond;
  return NTU_OK;
}

extern "C" int ntu_env_metric(ntu_ctx* c, int bond, double* g_out, double* diag_out) {
  if (!c) return fail(c, NTU_EINVAL, "NULL context");
  if (c->stage < 1 || c->stage_bond != bond)
    return fail(c, NTU_ESTATE, "ntu_env_metric(bond=%d) needs ntu_apply_gate on that bond first", bond);
  int st = cell_env(c);
  if (st) return st;
  if (g_out)
    CK(cudaMemcpyAsync(g_out, c->w.g, c->plan.szG * sizeof(double2), cudaMemcpyDeviceToHost,
                       c->stream), "copy g");
  if (diag_out)
    CK(cudaMemcpyAsync(diag_out, c->w.diag, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
       "copy diag");
  st = check_status(c);
  if (st) return st;
  c->stage = 2;
  return NTU_OK;
}

extern "C" int ntu_als_truncate(ntu_ctx* c, int bond, double* eps_out, double* delta_out,
                                double* tau_out) {
  if (!c) return fail(c, NTU_EINVAL, "NULL context");
  if (c->stage != 2 || c->stage_bond != bond)
    return fail(c, NTU_ESTATE, "ntu_als_truncate(bond=%d) needs ntu_env_metric on that bond first", bond);
  double* info_dev = c->w.info + 4 * (size_t)c->w.cap;
  int st = cell_als(c, bond, info_dev);
  if (st) return st;
  double info[4];
  CK(cudaMemcpyAsync(info, info_dev, sizeof(info), cudaMemcpyDeviceToHost, c->stream), "copy info");
  st = check_status(c);
  c->stage = 0;
  if (st) return st;
  if (eps_out) *eps_out = info[0];
  if (delta_out) *delta_out = info[1];
  if (tau_out) *tau_out = info[3];
  return NTU_OK;
}

static int su_bond(ntu_ctx* c, int bond, const double2* gate_dev, double* info_dev);

// The device work of one unit-cell Trotter step (NTU or SU bond updates),
// reading the gates from W.cG / W.op and writing the deltas to info_dev.
static int step_body(ntu_ctx* c, bool su, bool gate1, double* info_dev) {
  const Plan& P = c->plan;
  Work& W = c->w;
  const size_t d4 = (size_t)P.d * P.d * P.d * P.d;
  if (gate1) CK(launch_site_gate(c, W.A, W.B, W.op), "site gate");
  for (int b = 0; b < 4; ++b) {
    int st;
    if (su) {
      st = su_bond(c, b, W.cG + b * d4, info_dev + 4 * b);
    } else {
      st = cell_gate_qr(c, b, W.cG + b * d4);
      if (!st) st = cell_env(c);
      if (!st) st = cell_als(c, b, info_dev + 4 * b);
    }
    if (st) return st;
  }
  if (gate1) CK(launch_site_gate(c, W.A, W.B, W.op), "site gate");
  return NTU_OK;
}

// Runs step_body, through a CUDA graph captured on first use when graphs
// are on (one per form); falls back to direct launches where capture fails.
static int run_step(ntu_ctx* c, bool su, bool gate1, double* info_dev) {
  const int slot = (su ? 2 : 0) + (gate1 ? 1 : 0);
  if (c->use_graphs && !c->debug_sync && c->stream) {
    if (!c->step_graph[slot]) {
      cudaGraph_t g = nullptr;
      const int before = c->launches;
      if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
        int st = step_body(c, su, gate1, info_dev);
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (st == NTU_OK && e == cudaSuccess && g) {
          cudaGraphExec_t x = nullptr;
          if (cudaGraphInstantiate(&x, g, 0) == cudaSuccess) {
            c->step_graph[slot] = x;
            c->step_graph_launches[slot] = c->launches - before;
          }
        }
        if (g) cudaGraphDestroy(g);
        if (st != NTU_OK) return st;
      }
      cudaGetLastError();          // a refused capture leaves no sticky error
      c->launches = before;
    }
    if (c->step_graph[slot]) {
      CK(cudaGraphLaunch(c->step_graph[slot], c->stream), "graph launch");
      c->launches += c->step_graph_launches[slot];
      return NTU_OK;
    }
  }
  return step_body(c, su, gate1, info_dev);
}

extern "C" int ntu_step(ntu_ctx* c, const double* gates2, const double* gate1_half,
                        double* delta_out) {
  if (!c || !gates2) return fail(c, NTU_EINVAL, "ntu_step: NULL argument");
  const Plan& P = c->plan;
  Work& W = c->w;
  size_t d4 = (size_t)P.d * P.d * P.d * P.d, d2 = (size_t)P.d * P.d;
  CK(cudaMemcpyAsync(W.cG, gates2, 4 * d4 * sizeof(double2), cudaMemcpyHostToDevice, c->stream),
     "copy gates");
  if (gate1_half)
    CK(cudaMemcpyAsync(W.op, gate1_half, d2 * sizeof(double2), cudaMemcpyHostToDevice, c->stream),
       "copy gate1");
  double* info_dev = W.info + 4 * (size_t)W.cap;
  c->launches = 0;
  int st0 = run_step(c, false, gate1_half != nullptr, info_dev);
  if (st0) return st0;
  double info[16];
  CK(cudaMemcpyAsync(info, info_dev, sizeof(info), cudaMemcpyDeviceToHost, c->stream), "copy info");
  int st = check_status(c);
  c->stage = 0;
  if (st) return st;
  if (delta_out)
    for (int b = 0; b < 4; ++b) delta_out[b] = info[4 * b + 1];
  return NTU_OK;
}

extern "C" int ntu_measure(ntu_ctx* c, int site, const double* op, double* value_out) {
  if (!c || !op || !value_out) return fail(c, NTU_EINVAL, "ntu_measure: NULL argument");
  if (site < 0 || site > 1) return fail(c, NTU_EINVAL, "site=%d outside 0..1", site);
  const Plan& P = c->plan;
  Work& W = c->w;
  size_t d2 = (size_t)P.d * P.d;
  double2* opd = W.op + d2;
  CK(cudaMemcpyAsync(opd, op, d2 * sizeof(double2), cudaMemcpyHostToDevice, c->stream), "copy op");
  CK(launch_measure(c, site ? W.B : W.A, site ? W.A : W.B, opd, W.mval), "measure");
  CK(cudaMemcpyAsync(value_out, W.mval, sizeof(double2), cudaMemcpyDeviceToHost, c->stream),
     "copy value");
  return check_status(c);
}

// ------------------------------------------------ simple update (Sec. II)
extern "C" int ntu_su_set_lambdas(ntu_ctx* c, const double* lam) {
  if (!c || !lam) return fail(c, NTU_EINVAL, "ntu_su_set_lambdas: NULL argument");
  const int D = c->cfg.D;
  for (int i = 0; i < 4 * D; ++i)
    if (!(lam[i] >= 0.0) || !(lam[i] < INFINITY))
      return fail(c, NTU_EINVAL, "lambda[%d][%d] = %g is not a finite non-negative value", i / D,
                  i % D, lam[i]);
  CK(cudaMemcpyAsync(c->w.lam, lam, 4 * D * sizeof(double), cudaMemcpyHostToDevice, c->stream),
     "copy lambdas");
  return check_status(c);
}

extern "C" int ntu_su_get_lambdas(ntu_ctx* c, double* lam) {
  if (!c || !lam) return fail(c, NTU_EINVAL, "ntu_su_get_lambdas: NULL argument");
  CK(cudaMemcpyAsync(lam, c->w.lam, 4 * c->cfg.D * sizeof(double), cudaMemcpyDeviceToHost,
                     c->stream), "copy lambdas");
  return check_status(c);
}

// One SU bond update of the cell's state on the device (no synchronisation):
// weight the outer legs, orient, gate + QR, identity-metric truncation with
// zero sweeps, recompose, write back, unweight, new lambda_bond.
static int su_bond(ntu_ctx* c, int bond, const double2* gate_dev, double* info_dev) {
  Work& W = c->w;
  CK(launch_su_weight(c, bond, 0, 0, W.A, W.B, W.cA2, W.cB2), "SU weight");
  CK(launch_orient(c, bond, W.cA2, W.cB2, W.cTa, W.cTb), "orient");
  CK(launch_gate_qr(c, 1, W.cTa, W.cTb, gate_dev, bond >= 2 ? 1 : 0, W.QA, W.RA, W.QB, W.RB),
     "gate + QR");
  CK(launch_identity_metric(c, W.g), "identity metric");
  CK(launch_als(c, 1, W.g, W.RA, W.RB, W.MA, W.MB, info_dev, 0), "SU truncation");
  CK(launch_recompose(c, 1, W.QA, W.QB, W.MA, W.MB, W.cA2, W.cB2), "recompose");
  CK(launch_deorient(c, bond, W.cA2, W.cB2, W.A, W.B), "write back");
  CK(launch_su_weight(c, bond, 1, 1, W.A, W.B, W.A, W.B), "SU unweight");
  CK(launch_su_lambda(c, bond), "SU lambda");
  return NTU_OK;
}

extern "C" int ntu_su_update(ntu_ctx* c, int bond, const double* gate, double* delta_out) {
  if (!c || !gate) return fail(c, NTU_EINVAL, "ntu_su_update: NULL argument");
  if (bond < 0 || bond > 3) return fail(c, NTU_EINVAL, "bond=%d outside 0..3", bond);
  const Plan& P = c->plan;
  size_t d4 = (size_t)P.d * P.d * P.d * P.d;
  CK(cudaMemcpyAsync(c->w.cG, gate, d4 * sizeof(double2), cudaMemcpyHostToDevice, c->stream),
     "copy gate");
  double* info_dev = c->w.info + 4 * (size_t)c->w.cap;
  int st = su_bond(c, bond, c->w.cG, info_dev);
  if (st) return st;
  double info[4];
  CK(cudaMemcpyAsync(info, info_dev, sizeof(info), cudaMemcpyDeviceToHost, c->stream), "copy info");
  st = check_status(c);
  c->stage = 0;
  if (st) return st;
  if (delta_out) *delta_out = info[1];
  return NTU_OK;
}

extern "C" int ntu_su_step(ntu_ctx* c, const double* gates2, const double* gate1_half,
                           double* delta_out) {
  if (!c || !gates2) return fail(c, NTU_EINVAL, "ntu_su_step: NULL argument");
  const Plan& P = c->plan;
  Work& W = c->w;
  size_t d4 = (size_t)P.d * P.d * P.d * P.d, d2 = (size_t)P.d * P.d;
  CK(cudaMemcpyAsync(W.cG, gates2, 4 * d4 * sizeof(double2), cudaMemcpyHostToDevice, c->stream),
     "copy gates");
  if (gate1_half)
    CK(cudaMemcpyAsync(W.op, gate1_half, d2 * sizeof(double2), cudaMemcpyHostToDevice, c->stream),
       "copy gate1");
  double* info_dev = W.info + 4 * (size_t)W.cap;
  c->launches = 0;
  int st0 = run_step(c, true, gate1_half != nullptr, info_dev);
  if (st0) return st0;
  double info[16];
  CK(cudaMemcpyAsync(info, info_dev, sizeof(info), cudaMemcpyDeviceToHost, c->stream), "copy info");
  int st = check_status(c);
  c->stage = 0;
  if (st) return st;
  if (delta_out)
    for (int b = 0; b < 4; ++b) delta_out[b] = info[4 * b + 1];
  return NTU_OK;
}

// ---------------------------------------------------------------- batches
static int check_batch(ntu_ctx* c, int n) {
  if (!c) return fail(c, NTU_EINVAL, "NULL context");
  if (n < 0 || n > c->w.cap)
    return fail(c, NTU_EINVAL, "n=%d outside 0..max_batch=%d", n, c->w.cap);
  return NTU_OK;
}

extern "C" int ntu_batch_update_dev(ntu_ctx* c, int n, const double* Ta, const double* Tb,
                                    const double* gates, double* Ta_out, double* Tb_out,
                                    double* info) {
  int st = check_batch(c, n);
  if (st) return st;
  if (n == 0) return NTU_OK;
  if (!Ta || !Tb || !gates || !Ta_out || !Tb_out || !info)
    return fail(c, NTU_EINVAL, "ntu_batch_update_dev: NULL argument");
  Work& W = c->w;
  c->launches = 0;
  const bool prof = c->profiling != 0;
  const double2 *ta = (const double2*)Ta, *tb = (const double2*)Tb;
  if (prof) CK(cudaEventRecord(c->ev[0], c->stream), "event");
  CK(launch_gate_qr(c, n, ta, tb, (const double2*)gates, 0, W.QA, W.RA, W.QB, W.RB), "gate + QR");
  if (prof) CK(cudaEventRecord(c->ev[1], c->stream), "event");
  CK(launch_env(c, n, ta, tb, W.QA, W.QB, W.graw), "environment");
  if (prof) CK(cudaEventRecord(c->ev[2], c->stream), "event");
  CK(launch_repair(c, n, W.graw, c->cfg.precision != NTU_FP64, W.g, W.diag), "repair");
  if (prof) CK(cudaEventRecord(c->ev[3], c->stream), "event");
  CK(launch_als(c, n, W.g, W.RA, W.RB, W.MA, W.MB, info), "ALS");
  if (prof) CK(cudaEventRecord(c->ev[4], c->stream), "event");
  CK(launch_recompose(c, n, W.QA, W.QB, W.MA, W.MB, (double2*)Ta_out, (double2*)Tb_out),
     "recompose");
  if (prof) CK(cudaEventRecord(c->ev[5], c->stream), "event");
  return NTU_OK;
}

extern "C" int ntu_set_profiling(ntu_ctx* c, int on) {
  if (!c) return fail(c, NTU_EINVAL, "NULL context");
  if (on && !c->ev[0])
    for (int i = 0; i < 6; ++i) CK(cudaEventCreate(&c->ev[i]), "event create");
  c->profiling = on ? 1 : 0;
  return NTU_OK;
}

extern "C" int ntu_stage_times(ntu_ctx* c, double* ms_out) {
  if (!c || !ms_out) return fail(c, NTU_EINVAL, "ntu_stage_times: NULL argument");
  if (!c->profiling) return fail(c, NTU_ESTATE, "profiling is off");
  CK(cudaEventSynchronize(c->ev[5]), "event synchronize");
  for (int i = 0; i < 5; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]), "event elapsed");
    ms_out[i] = ms;
  }
  return NTU_OK;
}

// A host-buffer batch of at least two full ALS waves (2 x 3 x SMs items)
// runs as two halves: the second half's inputs are copied in on a second
// stream while the first half computes, and the first half's outputs are
// copied out while the second computes, so that only half of the copies
// stay outside the compute.  Each half keeps full ALS waves and the same
// kernels and schedule, so the results are those of one launch.
static int batch_update_host_halves(ntu_ctx* c, int n, const double* Ta, const double* Tb,
                                    const double* gates, double* Ta_out, double* Tb_out,
                                    double* info) {
  const Plan& P = c->plan;
  Work& W = c->w;
  if (!c->copy_stream) {
    CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking), "copy stream");
    for (int i = 0; i < 3; ++i)
      CK(cudaEventCreateWithFlags(&c->cev[i], cudaEventDisableTiming), "copy event");
  }
  cudaStream_t S = c->stream, C = c->copy_stream;
  const int n1 = n / 2, n2 = n - n1;
  const size_t t_item = (size_t)P.szT, g_item = (size_t)P.d * P.d * P.d * P.d;
  const size_t tb1 = n1 * t_item * sizeof(double2), tb2 = n2 * t_item * sizeof(double2);
  const size_t gb1 = n1 * g_item * sizeof(double2), gb2 = n2 * g_item * sizeof(double2);
  const size_t ot = n1 * t_item, og = n1 * g_item;      // element offsets of the second half
  // the second half's inputs go in on C only after S is past any earlier use
  // of the staging buffers
  CK(cudaEventRecord(c->cev[0], S), "event");
  CK(cudaStreamWaitEvent(C, c->cev[0], 0), "wait");
  CK(cudaMemcpyAsync(W.Ta_in, Ta, tb1, cudaMemcpyHostToDevice, S), "copy Ta");
  CK(cudaMemcpyAsync(W.Tb_in, Tb, tb1, cudaMemcpyHostToDevice, S), "copy Tb");
  CK(cudaMemcpyAsync(W.G_in, gates, gb1, cudaMemcpyHostToDevice, S), "copy gates");
  CK(cudaMemcpyAsync(W.Ta_in + ot, Ta + 2 * ot, tb2, cudaMemcpyHostToDevice, C), "copy Ta");
  CK(cudaMemcpyAsync(W.Tb_in + ot, Tb + 2 * ot, tb2, cudaMemcpyHostToDevice, C), "copy Tb");
  CK(cudaMemcpyAsync(W.G_in + og, gates + 2 * og, gb2, cudaMemcpyHostToDevice, C), "copy gates");
  CK(cudaEventRecord(c->cev[1], C), "event");
  int st = ntu_batch_update_dev(c, n1, (const double*)W.Ta_in, (const double*)W.Tb_in,
                                (const double*)W.G_in, (double*)W.Ta_out, (double*)W.Tb_out,
                                W.info);
  if (st) return st;
  CK(cudaEventRecord(c->cev[2], S), "event");
  CK(cudaStreamWaitEvent(C, c->cev[2], 0), "wait");
  CK(cudaMemcpyAsync(Ta_out, W.Ta_out, tb1, cudaMemcpyDeviceToHost, C), "copy Ta_out");
  CK(cudaMemcpyAsync(Tb_out, W.Tb_out, tb1, cudaMemcpyDeviceToHost, C), "copy Tb_out");
  CK(cudaMemcpyAsync(info, W.info, (size_t)n1 * 4 * sizeof(double), cudaMemcpyDeviceToHost, C),
     "copy info");
  CK(cudaStreamWaitEvent(S, c->cev[1], 0), "wait");
  st = ntu_batch_update_dev(c, n2, (const double*)(W.Ta_in + ot), (const double*)(W.Tb_in + ot),
                            (const double*)(W.G_in + og), (double*)(W.Ta_out + ot),
                            (double*)(W.Tb_out + ot), W.info + 4 * (size_t)n1);
  if (st) return st;
  CK(cudaMemcpyAsync(Ta_out + 2 * ot, W.Ta_out + ot, tb2, cudaMemcpyDeviceToHost, S),
     "copy Ta_out");
  CK(cudaMemcpyAsync(Tb_out + 2 * ot, W.Tb_out + ot, tb2, cudaMemcpyDeviceToHost, S),
     "copy Tb_out");
  CK(cudaMemcpyAsync(info + 4 * (size_t)n1, W.info + 4 * (size_t)n1,
                     (size_t)n2 * 4 * sizeof(double), cudaMemcpyDeviceToHost, S), "copy info");
  // the call returns when both streams are done
  CK(cudaEventRecord(c->cev[0], C), "event");
  CK(cudaStreamWaitEvent(S, c->cev[0], 0), "wait");
  return check_status(c);
}

extern "C" int ntu_batch_update_host(ntu_ctx* c, int n, const double* Ta, const double* Tb,
                                     const double* gates, double* Ta_out, double* Tb_out,
                                     double* info) {
  int st = check_batch(c, n);
  if (st) return st;
  if (n == 0) return NTU_OK;
  if (!Ta || !Tb || !gates || !Ta_out || !Tb_out || !info)
    return fail(c, NTU_EINVAL, "ntu_batch_update_host: NULL argument");
  if (n >= 6 * c->sms)
    return batch_update_host_halves(c, n, Ta, Tb, gates, Ta_out, Tb_out, info);
  const Plan& P = c->plan;
  Work& W = c->w;
  size_t tb = (size_t)n * P.szT * sizeof(double2);
  size_t gb = (size_t)n * P.d * P.d * P.d * P.d * sizeof(double2);
  CK(cudaMemcpyAsync(W.Ta_in, Ta, tb, cudaMemcpyHostToDevice, c->stream), "copy Ta");
  CK(cudaMemcpyAsync(W.Tb_in, Tb, tb, cudaMemcpyHostToDevice, c->stream), "copy Tb");
  CK(cudaMemcpyAsync(W.G_in, gates, gb, cudaMemcpyHostToDevice, c->stream), "copy gates");
  st = ntu_batch_update_dev(c, n, (const double*)W.Ta_in, (const double*)W.Tb_in,
                            (const double*)W.G_in, (double*)W.Ta_out, (double*)W.Tb_out, W.info);
  if (st) return st;
  CK(cudaMemcpyAsync(Ta_out, W.Ta_out, tb, cudaMemcpyDeviceToHost, c->stream), "copy Ta_out");
  CK(cudaMemcpyAsync(Tb_out, W.Tb_out, tb, cudaMemcpyDeviceToHost, c->stream), "copy Tb_out");
  CK(cudaMemcpyAsync(info, W.info, (size_t)n * 4 * sizeof(double), cudaMemcpyDeviceToHost,
                     c->stream), "copy info");
  return check_status(c);
}

extern "C" int ntu_batch_gate_qr_dev(ntu_ctx* c, int n, const double* Ta, const double* Tb,
                                     const double* gates, double* QA, double* RA, double* QB,
                                     double* RB) {
  int st = check_batch(c, n);
  if (st || n == 0) return st;
  if (!Ta || !Tb || !gates || !QA || !RA || !QB || !RB)
    return fail(c, NTU_EINVAL, "ntu_batch_gate_qr_dev: NULL argument");
  CK(launch_gate_qr(c, n, (const double2*)Ta, (const double2*)Tb, (const double2*)gates, 0,
                    (double2*)QA, (double2*)RA, (double2*)QB, (double2*)RB), "gate + QR");
  return NTU_OK;
}

extern "C" int ntu_batch_env_dev(ntu_ctx* c, int n, const double* Ta, const double* Tb,
                                 const double* QA, const double* QB, double* g) {
  int st = check_batch(c, n);
  if (st || n == 0) return st;
  if (!Ta || !Tb || !QA || !QB || !g) return fail(c, NTU_EINVAL, "ntu_batch_env_dev: NULL argument");
  if (c->cfg.precision == NTU_FP64) {
    CK(launch_env(c, n, (const double2*)Ta, (const double2*)Tb, (const double2*)QA,
                  (const double2*)QB, g), "environment");
  } else {
    CK(launch_env(c, n, (const double2*)Ta, (const double2*)Tb, (const double2*)QA,
                  (const double2*)QB, c->w.graw), "environment");
    CK(launch_copy_raw(c, n, c->w.graw, (double2*)g), "widen g");
  }
  return NTU_OK;
}

extern "C" int ntu_batch_repair_dev(ntu_ctx* c, int n, double* g, double* diag) {
  int st = check_batch(c, n);
  if (st || n == 0) return st;
  if (!g || !diag) return fail(c, NTU_EINVAL, "ntu_batch_repair_dev: NULL argument");
  CK(cudaMemcpyAsync(c->w.graw, g, (size_t)n * c->plan.szG * sizeof(double2),
                     cudaMemcpyDeviceToDevice, c->stream), "stage g");
  CK(launch_repair(c, n, c->w.graw, 0, (double2*)g, diag), "repair");
  return NTU_OK;
}

extern "C" int ntu_batch_als_dev(ntu_ctx* c, int n, const double* g, const double* RA,
                                 const double* RB, double* MA, double* MB, double* info) {
  int st = check_batch(c, n);
  if (st || n == 0) return st;
  if (!g || !RA || !RB || !MA || !MB || !info) return fail(c, NTU_EINVAL, "ntu_batch_als_dev: NULL argument");
  CK(launch_als(c, n, (const double2*)g, (const double2*)RA, (const double2*)RB, (double2*)MA,
                (double2*)MB, info), "ALS");
  return NTU_OK;
}

extern "C" int ntu_batch_recompose_dev(ntu_ctx* c, int n, const double* QA, const double* QB,
                                       const double* MA, const double* MB, double* Ta_out,
                                       double* Tb_out) {
  int st = check_batch(c, n);
  if (st || n == 0) return st;
  if (!QA || !QB || !MA || !MB || !Ta_out || !Tb_out)
    return fail(c, NTU_EINVAL, "ntu_batch_recompose_dev: NULL argument");
  CK(launch_recompose(c, n, (const double2*)QA, (const double2*)QB, (const double2*)MA,
                      (const double2*)MB, (double2*)Ta_out, (double2*)Tb_out), "recompose");
  return NTU_OK;
}
