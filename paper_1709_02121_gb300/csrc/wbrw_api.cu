// wbrw_api.cu -- the C ABI of include/wbrw.h: argument checks, the carve-up
// of the caller's scratch buffer, the resampling schedule of Sec. 4.3 and
// the state machine between "particles in the arrays" and "histogram".
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <new>
#include <vector>

#include "wbrw.h"
#include "wbrw_internal.h"

using namespace wbrw;

struct wbrw_ctx : public Ctx {};

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }


struct Layout {
  size_t counters, cpid, fq0, fq1, eq0, eq1, dq0, dq1, nz_cell, nz_start, tile_nz, scan_bsum,
      scan_bnz, tmp_grid, tmp_wsum, obs_density, obs_marg, obs_col, obs_scalar, rec_cell,
      rec_a, keep0, keep1, res0, res1, ucnt, guide, binst, dpre, bguide, seg_counts, cnt_save, tabs,
      cinst, obs_red, tab_A, tab_xmax, tab_xi0, tab_xi1, tab_cdf0, tab_cdf1, tab_guide0,
      tab_guide1, dgrid0, dgrid1, tnz_cell, tnz_start, tnz_tau, ttile_nz, total;
  long long qcap, ecap, dcap, rec_cap, scan_blocks, tile_cap;
};

// ninst = 0: a plain run (config->n_alpha is used); ninst >= 1: a batch.
bool config_ok(const wbrw_config* c, char* why, size_t n, int ninst = 0) {
  auto fail = [&](const char* m) {
    if (why) snprintf(why, n, "invalid configuration: %s", m);
    return false;
  };
  if (!c) return fail("NULL config");
  if (c->dim != 2 && c->dim != 4) return fail("dim must be 2 or 4");
  if (c->dim == 4 && c->strategy != WBRW_SP1_PAIR) return fail("dim 4 uses sp1 only");
  if (c->tangent != 0 && c->tangent != 1) return fail("tangent must be 0 or 1");
  if (c->tangent && (c->dim != 2 || c->strategy != WBRW_SP1_PAIR))
    return fail("tangents need dim 2 and sp1");
  if (c->tangent && !(c->tangent_quantum < 1e9)) return fail("tangent quantum");
  if (c->dim == 4 && ninst > 1) return fail("dim 4 runs one instance");
  if (c->table_ny < 0 || c->table_ny == 1 || c->table_nkappa < 0 || c->table_ny > (1 << 20) ||
      c->table_nkappa > (1 << 20))
    return fail("table sizes");
  if (c->precision != WBRW_FP64 && c->precision != WBRW_FP32) return fail("precision");
  if (c->strategy != WBRW_SP1_PAIR && c->strategy != WBRW_SP2_BOOTSTRAP &&
      c->strategy != WBRW_WP)
    return fail("strategy");
  if (!(c->hbar > 0) || !(c->mass > 0) || !(c->dt > 0)) return fail("hbar, mass and dt must be > 0");
  if (c->nx <= 0 || c->nk <= 0) return fail("nx and nk must be > 0");
  if (ninst < 0 || ninst > kMaxInst) return fail("instances must be 1..WBRW_MAX_INSTANCES");
  const long long cells = c->dim == 4 ? (long long)c->nx * c->nx * c->nk * c->nk
                                      : (long long)c->nx * c->nk;
  if (c->dim == 4 && (c->nx > 4096 || c->nk > 4096)) return fail("nx, nk <= 4096 for dim 4");
  if (cells * (ninst > 0 ? ninst : 1) >= (1ll << 30))
    return fail("cells of all instances must be < 2^30");
  if (!(c->xmax > c->xmin) || !(c->kmax > c->kmin)) return fail("empty domain");
  if (c->resample_every < 0) return fail("resample_every must be >= 0");
  if (ninst == 0 && c->n_alpha <= 0) return fail("n_alpha must be > 0");
  return true;
}

// Queue entries: {u64 pid; T x, k, w; int l;} (plus the tangent weights in
// the tangent mode) for offspring waves (FP64) and candidate intervals;
// deferred segments take 64 bytes (FP64 tangent mode: 80).  Every queue is cut
// into one segment per producer warp (at most kMaxSeg); each segment gets at
// least kMinSeg entries so that small runs cannot starve a warp.
constexpr long long kMinSeg = 64;
const Driver* drv_for(int precision, int dim, int tangent) {
  if (dim == 4) return precision == WBRW_FP64 ? driver_fp64_4d() : driver_fp32_4d();
  if (tangent) return precision == WBRW_FP64 ? driver_fp64_grad() : driver_fp32_grad();
  return precision == WBRW_FP64 ? driver_fp64() : driver_fp32();
}

// The tangent quantum in units of 2^-32 (at least one unit).
long long tquantum_of(const wbrw_config* c) {
  const double q = c->tangent_quantum > 0 ? c->tangent_quantum : 1.0;
  const double u = std::ldexp(q, 32);
  return u < 1.0 ? 1 : (long long)std::llround(u);
}

int table_ny(const wbrw_config* c) { return c->table_ny > 0 ? c->table_ny : 4096; }
int table_nkappa(const wbrw_config* c) { return c->table_nkappa > 0 ? c->table_nkappa : 2048; }

Layout layout(const wbrw_config* c, int ninst, long long capacity) {
  Layout L;
  const Driver* d = drv_for(c->precision, c->dim, c->tangent);
  const long long cells = c->dim == 4 ? (long long)c->nx * c->nx * c->nk * c->nk
                                      : (long long)c->nx * c->nk;
  const long long nh = cells * ninst;
  const long long floor_entries = (long long)kMaxSeg * kMinSeg;
  L.qcap = capacity > floor_entries ? capacity : floor_entries;
  // per round buffer: FP32 flights queue at most one candidate interval per
  // particle, FP64 flights all of them (about one per particle per flight)
  L.ecap = c->precision == WBRW_FP32 ? L.qcap : 2 * L.qcap;
  L.dcap = L.ecap / 4;  // deferred segments: a few per cent of the events
  L.tile_cap = capacity / 32 + 2;
  L.rec_cap = c->strategy == WBRW_SP2_BOOTSTRAP ? 4 * L.qcap : 0;
  L.scan_blocks = (nh + kScanTile - 1) / kScanTile;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  L.counters = take(sizeof(Counters));
  L.seg_counts = take((size_t)(2 + 2 + kMaxLevels + 1) * kMaxSeg * sizeof(unsigned));
  L.cnt_save = take(sizeof(Counters));
  L.cpid = take((size_t)capacity * 8);
  L.fq0 = take((size_t)L.qcap * d->fentry_bytes);
  L.fq1 = take((size_t)L.qcap * d->fentry_bytes);
  L.eq0 = take((size_t)L.ecap * d->fentry_bytes);
  L.eq1 = take((size_t)L.ecap * d->fentry_bytes);
  L.dq0 = take((size_t)L.dcap * d->sentry_bytes);
  L.dq1 = take((size_t)L.dcap * d->sentry_bytes);
  L.nz_cell = take((size_t)nh * 4);
  L.nz_start = take((size_t)nh * 8);
  L.tile_nz = take((size_t)L.tile_cap * 4);
  L.scan_bsum = take((size_t)(L.scan_blocks + 1) * 8);
  L.scan_bnz = take((size_t)(L.scan_blocks + 1) * 4);
  L.tmp_grid = take((size_t)nh * 4);
  L.tmp_wsum = take((size_t)nh * 8);
  L.obs_density = take((size_t)c->nx * c->nk * 8);
  L.obs_marg = take((size_t)c->nx * 8);
  L.obs_col = take((size_t)c->nx * 8);
  L.obs_scalar = take(64);
  L.obs_red = take(c->dim == 4 ? (size_t)c->nx * c->nk * 8 : 0);
  L.rec_cell = take((size_t)L.rec_cap * 4);
  L.rec_a = take((size_t)L.rec_cap * 4);
  const bool sp2 = c->strategy == WBRW_SP2_BOOTSTRAP;
  L.keep0 = take(sp2 ? (size_t)nh * 4 : 0);
  L.keep1 = take(sp2 ? (size_t)nh * 4 : 0);
  L.res0 = take(sp2 ? (size_t)nh * 8 : 0);
  L.res1 = take(sp2 ? (size_t)nh * 8 : 0);
  L.ucnt = take(sp2 ? (size_t)2 * nh * 4 : 0);
  L.guide = take(sp2 ? (size_t)2 * (kGuide + 1) * 4 : 0);
  L.binst = take(sp2 && ninst > 1 ? (size_t)ninst * sizeof(BootInst) : 0);
  L.dpre = take(sp2 && ninst > 1 ? (size_t)(2 * ninst + 1) * 8 : 0);
  L.bguide = take(sp2 && ninst > 1 ? (size_t)2 * ninst * (kGuideB + 1) * 4 : 0);
  L.tabs = take(kTabBytes);
  L.cinst = take(ninst > 1 ? (size_t)capacity * 4 : 0);
  const bool d4 = c->dim == 4;
  const size_t el = c->precision == WBRW_FP64 ? 8 : 4;
  const size_t ny = (size_t)table_ny(c), nk = (size_t)table_nkappa(c);
  L.tab_A = take(d4 ? 2 * nk * 8 : 0);
  L.tab_xmax = take(d4 ? 16 : 0);
  L.tab_xi0 = take(d4 ? ny * el : 0);
  L.tab_xi1 = take(d4 ? ny * el : 0);
  L.tab_cdf0 = take(d4 ? ny * nk * el : 0);
  L.tab_cdf1 = take(d4 ? ny * nk * el : 0);
  const size_t ng = d4 && el == 4 ? ny * (kTabGuide + 1) * 4 : 0;
  L.tab_guide0 = take(ng);
  L.tab_guide1 = take(ng);
  const bool tg = c->tangent != 0;
  L.dgrid0 = take(tg ? (size_t)nh * 8 : 0);
  L.dgrid1 = take(tg ? (size_t)nh * 8 : 0);
  L.tnz_cell = take(tg ? (size_t)nh * 4 : 0);
  L.tnz_start = take(tg ? (size_t)nh * 8 : 0);
  L.tnz_tau = take(tg ? (size_t)nh * 16 : 0);
  L.ttile_nz = take(tg ? (size_t)L.tile_cap * 4 : 0);
  L.total = off;
  return L;
}

// Constants of one instance (Sec. 4.2 / Remark 3 / Sec. 3.2): C = 2|H|/hbar,
// kick scale 1/(2w), rate gamma0 (default C/2), acceptance factor
// C/(2 gamma0) <= 1, P(candidate in an interval) = 1 - exp(-gamma0 dt).
bool make_instance(const wbrw_config* cfg, const wbrw_potential* pot, double gamma0_in,
                   double x0, double sx, double k0, long long n_init, long long n_alpha,
                   InstHost* q) {
  if (!pot || pot->kind != WBRW_POT_GAUSSIAN || !(pot->w > 0) || !isfinite(pot->w) ||
      !isfinite(pot->H) || !isfinite(pot->xc))
    return false;
  if (!(sx > 0) || !isfinite(sx) || !isfinite(x0) || !isfinite(k0)) return false;
  if (n_init < 0 || n_alpha <= 0) return false;
  q->H = pot->H;
  q->w = pot->w;
  q->xc = pot->xc;
  q->C = 2.0 * fabs(pot->H) / cfg->hbar;
  double g = gamma0_in > 0 ? gamma0_in : 0.5 * q->C;
  if (g <= 0) g = 1.0;  // H = 0: no pair is ever accepted
  q->gamma0 = g;
  q->cacc = q->C / (2.0 * g);
  if (q->cacc > 1.0) return false;  // gamma0 below the majorant rate C/2
  q->sig_k = 1.0 / (2.0 * pot->w);
  q->p_any = -expm1(-g * cfg->dt);
  q->x0 = x0;
  q->sx = sx;
  q->k0 = k0;
  q->n_init = n_init;
  q->n_alpha = n_alpha;
  q->start = 0;
  return true;
}

void free_ctx(wbrw_ctx* c) {
  if (!c) return;
  free(c->ih);
  free(c->host_tab);
  delete c;
}

wbrw_status seterr(wbrw_ctx* c, wbrw_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(c->err, sizeof(c->err), fmt, ap);
  va_end(ap);
  if (st != WBRW_ERR_ARG) c->failed = 1;
  return st;
}

wbrw_status cuda_check(wbrw_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return WBRW_OK;
  return seterr(c, WBRW_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

const Driver* drv(const wbrw_ctx* c) {
  if (c->lean) {
    if (c->cfg.tangent) return driver_fp32_grad_lean();
    return c->ninst > 1 ? driver_fp32_lean_batch() : driver_fp32_lean();
  }
  return drv_for(c->cfg.precision, c->cfg.dim, c->cfg.tangent);
}

#define WBRW_TRY(c, expr, what)                           \
  do {                                                    \
    wbrw_status st_ = cuda_check((c), (expr), (what));    \
    if (st_ != WBRW_OK) return st_;                       \
  } while (0)

// Translate the device error word.
wbrw_status device_status(wbrw_ctx* c) {
  int err = 0;
  WBRW_TRY(c, cudaMemcpyAsync(&err, &c->cnt->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
           "read device error word");
  WBRW_TRY(c, cudaStreamSynchronize(c->stream), "synchronise");
  if (err == 0) return WBRW_OK;
  return seterr(c, (err & ERR_NUMERIC) ? WBRW_ERR_NUMERIC : WBRW_ERR_CAPACITY,
                "device error 0x%x:%s%s%s%s%s%s", err,
                (err & ERR_NUMERIC) ? " non-finite position or wavevector at binning;" : "",
                (err & ERR_CAP_PARTICLES) ? " particle capacity exceeded;" : "",
                (err & ERR_CAP_QUEUE) ? " offspring queue capacity exceeded;" : "",
                (err & ERR_CAP_EQUEUE) ? " candidate queue capacity exceeded;" : "",
                (err & ERR_NESTING) ? " offspring nesting within one interval too deep;" : "",
                (err & ERR_CAP_RECORDS) ? " bootstrap record capacity exceeded;" : "");
}

cudaError_t zero_tangent(wbrw_ctx* c) {
  cudaError_t e = launch_zero(c, c->dgrid[0], (size_t)c->nh * 8);
  return e == cudaSuccess ? launch_zero(c, c->dgrid[1], (size_t)c->nh * 8) : e;
}

// Histogram the particles of the arrays into c->buf.grid (sp1) or run the
// signed bootstrap (sp2), then build the regeneration plan.  c->epoch has
// already been advanced.
wbrw_status resample_from_arrays(wbrw_ctx* c) {
  const Driver* d = drv(c);
  if (c->cfg.strategy == WBRW_SP1_PAIR) {
    WBRW_TRY(c, launch_zero(c, c->buf.grid, (size_t)c->nh * 4), "zero grid");
    if (c->tangent) WBRW_TRY(c, zero_tangent(c), "zero tangent");
    WBRW_TRY(c, d->bin(c, DST_BIN1, c->buf.grid, 1), "bin");
  } else if (c->cfg.strategy == WBRW_WP) {
    WBRW_TRY(c, launch_zero(c, c->tmp_wsum, (size_t)c->nh * 8), "zero");
    WBRW_TRY(c, d->bin(c, DST_WSUM, c->buf.grid, 1), "weights");
    WBRW_TRY(c, launch_wp_round(c, 0), "rounding");  // binning set the new epoch's id base
  } else {
    WBRW_TRY(c, launch_setup(c, SETUP_BOOT, 0, 0), "setup");
    WBRW_TRY(c, launch_zero(c, c->rcnt, (size_t)c->nseg * sizeof(unsigned)), "zero");
    WBRW_TRY(c, launch_zero(c, c->boot_ucnt, (size_t)2 * c->nh * 4), "zero");
    WBRW_TRY(c, d->bin(c, DST_BIN2, c->buf.grid, 1), "records");
    WBRW_TRY(c, launch_boot(c, 0), "bootstrap");
  }
  WBRW_TRY(c, launch_scan_cells(c, c->buf.grid), "scan");
  if (c->tangent) WBRW_TRY(c, launch_scan_tangent(c), "tangent plan");
  return WBRW_OK;
}

// One fused period of wbrw_run: zero the histogram (sp1) or the bootstrap
// tallies (sp2), fly [l0, L) from src into the sink, bootstrap (sp2), and
// build the regeneration plan.  The source's ids are those of regen_epoch;
// the histogram made here is epoch regen_epoch + 1, which c->epoch holds on
// return.
wbrw_status enqueue_period(wbrw_ctx* c, int src, int l0, int L, long long regen_epoch) {
  const Driver* d = drv(c);
  c->epoch = regen_epoch + 1;
  if (c->cfg.strategy == WBRW_SP1_PAIR) {
    WBRW_TRY(c, launch_zero(c, c->buf.grid, (size_t)c->nh * 4), "zero grid");
    if (c->tangent) WBRW_TRY(c, zero_tangent(c), "zero tangent");
  } else if (c->cfg.strategy == WBRW_WP) {
    WBRW_TRY(c, launch_zero(c, c->tmp_wsum, (size_t)c->nh * 8), "zero");
  } else {
    WBRW_TRY(c, launch_setup(c, SETUP_BOOT, 0, 0), "setup");
    WBRW_TRY(c, launch_zero(c, c->rcnt, (size_t)c->nseg * sizeof(unsigned)), "zero");
    WBRW_TRY(c, launch_zero(c, c->boot_ucnt, (size_t)2 * c->nh * 4), "zero");
  }
  // the regeneration of the previous histogram uses its own epoch's ids
  const long long keep_epoch = c->epoch;
  c->epoch = regen_epoch;
  const int dst = c->cfg.strategy == WBRW_SP1_PAIR ? DST_BIN1
                  : (c->cfg.strategy == WBRW_WP ? DST_WSUM : DST_BIN2);
  cudaError_t e = d->chunk(c, l0, L, src, dst);
  c->epoch = keep_epoch;
  WBRW_TRY(c, e, "period");
  // the device id base is still the source's epoch: the histogram is the next
  if (c->cfg.strategy == WBRW_SP2_BOOTSTRAP) WBRW_TRY(c, launch_boot(c, 1), "bootstrap");
  if (c->cfg.strategy == WBRW_WP) WBRW_TRY(c, launch_wp_round(c, 1), "rounding");
  WBRW_TRY(c, launch_scan_cells(c, c->buf.grid), "scan");
  if (c->tangent) WBRW_TRY(c, launch_scan_tangent(c), "tangent plan");
  return WBRW_OK;
}

void drop_graphs(wbrw_ctx* c) {
  for (int i = 0; i < c->ngraphs; ++i) {
    if (c->graphs[i].exec) cudaGraphExecDestroy(c->graphs[i].exec);
    if (c->graphs[i].graph) cudaGraphDestroy(c->graphs[i].graph);
  }
  c->ngraphs = 0;
}

// Capture one period of length len that regenerates from the histogram.
// Its kernels take the first interval and the id base from the device
// period state, which the graph advances at its end.
wbrw_status capture_period(wbrw_ctx* c, int len, PeriodGraph* g) {
  memset(g, 0, sizeof(*g));
  g->len = len;
  g->prof = c->prof_on;
  const long long launches0 = c->launches;
  const long long epoch0 = c->epoch;
  WBRW_TRY(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal),
           "begin capture");
  c->capturing = 1;
  wbrw_status st = enqueue_period(c, SRC_REGEN, (int)c->step, (int)c->step + len, c->epoch);
  if (st == WBRW_OK)
    st = cuda_check(c, launch_setup(c, SETUP_ADVANCE, (unsigned long long)len, 0), "advance");
  if (c->prof_side_used) {  // join the profiling branch before the capture ends
    cudaEventRecord(c->prof_join, c->prof_side);
    cudaStreamWaitEvent(c->stream, c->prof_join, 0);
    c->prof_side_used = 0;
  }
  c->capturing = 0;
  c->epoch = epoch0;
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
  g->launches = c->launches - launches0;
  c->launches = launches0;
  if (st != WBRW_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  WBRW_TRY(c, e, "end capture");
  g->graph = graph;
  size_t n = 0;
  WBRW_TRY(c, cudaGraphGetNodes(graph, nullptr, &n), "graph nodes");
  cudaGraphNode_t* nodes = (cudaGraphNode_t*)calloc(n ? n : 1, sizeof(cudaGraphNode_t));
  if (!nodes) return seterr(c, WBRW_ERR_ARG, "out of host memory");
  cudaError_t ge = cudaGraphGetNodes(graph, nodes, &n);
  for (size_t i = 0; ge == cudaSuccess && i < n; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) != cudaSuccess || t != cudaGraphNodeTypeEventRecord)
      continue;
    cudaEvent_t ev;
    if (cudaGraphEventRecordNodeGetEvent(nodes[i], &ev) != cudaSuccess) continue;
    if (ev == c->gev[0]) g->ev_begin = nodes[i];
    if (ev == c->gev[1]) g->ev_end = nodes[i];
    for (int r = 0; r < kProfRounds; ++r) {
      if (ev == c->gev[2 + 2 * r]) g->evk_begin[r] = nodes[i];
      if (ev == c->gev[3 + 2 * r]) g->evk_end[r] = nodes[i];
    }
  }
  free(nodes);
  while (g->nevk < kProfRounds && g->evk_begin[g->nevk] && g->evk_end[g->nevk]) g->nevk += 1;
  WBRW_TRY(c, ge, "graph nodes");
  WBRW_TRY(c, cudaGraphInstantiate(&g->exec, graph, 0), "instantiate graph");
  return WBRW_OK;
}

// Replay (capturing first if needed) one regenerating period.
wbrw_status graph_period(wbrw_ctx* c, int len) {
  PeriodGraph* g = nullptr;
  for (int i = 0; i < c->ngraphs; ++i)
    if (c->graphs[i].len == len) g = &c->graphs[i];
  if (g && g->prof != c->prof_on) {  // profiling switched: capture again
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    wbrw_status st = capture_period(c, len, g);
    if (st != WBRW_OK) {
      if (g->exec) cudaGraphExecDestroy(g->exec);
      if (g->graph) cudaGraphDestroy(g->graph);
      *g = c->graphs[c->ngraphs - 1];
      c->ngraphs -= 1;
      return st;
    }
  }
  if (!g) {
    if (c->ngraphs == kMaxGraphs) drop_graphs(c);
    g = &c->graphs[c->ngraphs];
    wbrw_status st = capture_period(c, len, g);
    if (st != WBRW_OK) return st;
    c->ngraphs += 1;
  }
  if (!c->dev_period_ok)
    WBRW_TRY(c, launch_setup(c, SETUP_PERIOD, (unsigned long long)c->step,
                             (unsigned long long)c->epoch << 40), "period state");
  if (g->ev_begin && g->ev_end) {
    const bool on = c->prof_on && c->prof_n < kProfLaunches;
    WBRW_TRY(c, cudaGraphExecEventRecordNodeSetEvent(
                    g->exec, g->ev_begin, on ? c->prof_ev[2 * c->prof_n] : c->gev[0]),
             "profile event");
    WBRW_TRY(c, cudaGraphExecEventRecordNodeSetEvent(
                    g->exec, g->ev_end, on ? c->prof_ev[2 * c->prof_n + 1] : c->gev[1]),
             "profile event");
    if (on) c->prof_n += 1;
  }
  // the event kernel's records: on profiling events while profiling, else
  // back on the placeholders (once)
  const bool on_k = c->prof_on && c->prof_nk + g->nevk <= kProfLaunches;
  if (on_k || g->evk_live) {
    for (int r = 0; r < g->nevk; ++r) {
      WBRW_TRY(c, cudaGraphExecEventRecordNodeSetEvent(
                      g->exec, g->evk_begin[r],
                      on_k ? c->prof_evk[2 * (c->prof_nk + r)] : c->gev[2 + 2 * r]),
               "profile event");
      WBRW_TRY(c, cudaGraphExecEventRecordNodeSetEvent(
                      g->exec, g->evk_end[r],
                      on_k ? c->prof_evk[2 * (c->prof_nk + r) + 1] : c->gev[3 + 2 * r]),
               "profile event");
    }
    if (on_k) c->prof_nk += g->nevk;
    g->evk_live = on_k ? 1 : 0;
  }
  WBRW_TRY(c, cudaGraphLaunch(g->exec, c->stream), "graph launch");
  c->launches += g->launches;
  return WBRW_OK;
}

wbrw_status ensure_particles(wbrw_ctx* c) {
  if (c->state == ST_PARTICLES) return WBRW_OK;
  WBRW_TRY(c, drv(c)->materialize(c), "regenerate");
  c->state = ST_PARTICLES;
  return WBRW_OK;
}

wbrw_status step_impl(wbrw_ctx* c, int nsteps) {
  wbrw_status st = ensure_particles(c);
  if (st != WBRW_OK) return st;
  while (nsteps > 0) {
    const int ch = nsteps < c->max_chunk ? nsteps : c->max_chunk;
    WBRW_TRY(c, drv(c)->chunk(c, (int)c->step, (int)c->step + ch, SRC_ARRAY, DST_ARRAY), "step");
    c->step += ch;
    nsteps -= ch;
    c->fresh = 0;
  }
  return WBRW_OK;
}

}  // namespace

namespace wbrw {
// While a period is captured the pair becomes two event-record nodes on
// placeholder events (one pair per round for the event kernel); each replay
// points them at the profiling events.  Captured or not, the records sit on
// a side stream that waits for the stream's work so far: a record in the
// stream's own order delays the next kernel by several microseconds.
static void side_record(Ctx* c, cudaEvent_t ev) {
  cudaEventRecord(c->prof_fork, c->stream);
  cudaStreamWaitEvent(c->prof_side, c->prof_fork, 0);
  if (c->capturing) {
    cudaEventRecordWithFlags(ev, c->prof_side, cudaEventRecordExternal);
    c->prof_side_used = 1;
  } else {
    cudaEventRecord(ev, c->prof_side);
  }
}

void prof_begin(Ctx* c, int kind, int r) {
  if (c->capturing) {
    if (!c->prof_on) return;
    if (kind == PROF_FIRST_WAVE)
      side_record(c, c->gev[0]);
    else if (r < kProfRounds)
      side_record(c, c->gev[2 + 2 * r]);
    return;
  }
  if (!c->prof_on) return;
  if (kind == PROF_FIRST_WAVE) {
    if (c->prof_n < kProfLaunches) side_record(c, c->prof_ev[2 * c->prof_n]);
  } else if (c->prof_nk < kProfLaunches) {
    side_record(c, c->prof_evk[2 * c->prof_nk]);
  }
}
void prof_end(Ctx* c, int kind, int r) {
  if (c->capturing) {
    if (!c->prof_on) return;
    if (kind == PROF_FIRST_WAVE)
      side_record(c, c->gev[1]);
    else if (r < kProfRounds)
      side_record(c, c->gev[3 + 2 * r]);
    return;
  }
  if (!c->prof_on) return;
  if (kind == PROF_FIRST_WAVE) {
    if (c->prof_n < kProfLaunches) side_record(c, c->prof_ev[2 * c->prof_n + 1]);
    c->prof_n += c->prof_n < kProfLaunches;
  } else if (c->prof_nk < kProfLaunches) {
    side_record(c, c->prof_evk[2 * c->prof_nk + 1]);
    c->prof_nk += 1;
  }
}
}  // namespace wbrw

extern "C" {

size_t wbrw_scratch_bytes(const wbrw_config* config, long long capacity) {
  if (!config_ok(config, nullptr, 0) || capacity <= 0) return 0;
  return layout(config, 1, capacity).total;
}

size_t wbrw_batch_scratch_bytes(const wbrw_config* config, int ninst, long long capacity) {
  if (ninst < 1 || !config_ok(config, nullptr, 0, ninst) || capacity <= 0) return 0;
  return layout(config, ninst, capacity).total;
}

}  // extern "C"

namespace {

// Resident blocks per SM of the queue kernels, and with it the queue
// segmentation: one segment per warp of the grid.
void set_shape(wbrw_ctx* c, int bps) {
  c->bps = bps;
  c->nseg = bps * c->num_sms * (kBlock / 32);
  if (c->nseg > kMaxSeg) c->nseg = kMaxSeg;
  c->qseg = c->qcap / c->nseg;
  c->eseg = c->ecap / c->nseg;
  c->dseg = c->dcap / c->nseg;
  c->rseg = c->rec_cap / c->nseg;
}

// The 4D model's kernel tables: A_tj = (4 q_t / (pi hbar)) K0(2 a |kappa_j|)
// on the host (the library routine for K0), rows and running sums on the
// device; then each component's rate, the smallest multiple of 2^-10 at or
// above its largest xi, and the total rate Gamma = 2 gamma_0 + gamma_1 of the
// candidate clock (one-body terms on electrons 1 and 2, and the interaction).
wbrw_status build_tables(wbrw_ctx* c, char* base, const Layout& L) {
  const wbrw_config& g = c->cfg;
  c->tab_ny = table_ny(&g);
  c->tab_nkap = table_nkappa(&g);
  c->tab_K = g.kmax - g.kmin;
  c->tab_dkap = 2.0 * c->tab_K / (double)c->tab_nkap;
  for (int t = 0; t < 2; ++t) {
    c->tab_Y[t] = t == 0 ? (g.xmax - g.xmin) : 2.0 * (g.xmax - g.xmin);
    c->tab_dy[t] = 2.0 * c->tab_Y[t] / (double)(c->tab_ny - 1);
    c->tab_inv_dy[t] = (double)(c->tab_ny - 1) / (2.0 * c->tab_Y[t]);
  }
  c->tab_A = (double*)(base + L.tab_A);
  c->tab_xmax = (unsigned long long*)(base + L.tab_xmax);
  c->tab_xi[0] = base + L.tab_xi0;
  c->tab_xi[1] = base + L.tab_xi1;
  c->tab_cdf[0] = base + L.tab_cdf0;
  c->tab_cdf[1] = base + L.tab_cdf1;
  c->tab_guide[0] = (int*)(base + L.tab_guide0);
  c->tab_guide[1] = (int*)(base + L.tab_guide1);
  std::vector<double> A((size_t)2 * c->tab_nkap);
  const double pi = 3.141592653589793238462643383280;
  for (int t = 0; t < 2; ++t) {
    const double q = t == 0 ? -c->pot.H : c->pot.ee;
    const double pre = (4.0 * q) / (pi * g.hbar);
    for (int j = 0; j < c->tab_nkap; ++j) {
      const double kap = -c->tab_K + ((double)j + 0.5) * c->tab_dkap;
      A[(size_t)t * c->tab_nkap + j] = pre * std::cyl_bessel_k(0.0, 2.0 * c->pot.w * fabs(kap));
    }
  }
  double xmax[2] = {0, 0};
  WBRW_TRY(c, drv(c)->tables(c, A.data(), xmax), "kernel tables");
  for (int t = 0; t < 2; ++t) c->tab_gam[t] = ceil(1024.0 * xmax[t]) / 1024.0;
  InstHost& q = c->ih[0];
  double Gam = 2.0 * c->tab_gam[0] + c->tab_gam[1];
  if (!(Gam > 0)) Gam = 1.0;  // no potential: no pair is ever made
  q.gamma0 = Gam;
  q.cacc = 1.0;
  q.sig_k = 0.0;
  q.C = 0.0;
  q.p_any = -expm1(-Gam * g.dt);
  return WBRW_OK;
}

// Create a context for ninst instances (records q, starts filled in here)
// and enqueue the initial sampling.  Takes ownership of q.
wbrw_status create(const wbrw_config* config, const wbrw_potential* pot, int ninst, InstHost* q,
                   const wbrw_buffers* b, void* cuda_stream, wbrw_ctx** out, int ncomp = 0,
                   const Comp* comps = nullptr) {
  const long long cells = config->dim == 4
                              ? (long long)config->nx * config->nx * config->nk * config->nk
                              : (long long)config->nx * config->nk;
  if (!b || !b->x || !b->k || !b->s || !b->grid || !b->scratch || b->capacity <= 0 ||
      b->capacity > WBRW_MAX_CAPACITY ||
      (config->strategy != WBRW_SP1_PAIR && !b->w) ||
      b->grid_cells < cells * ninst || (config->tangent && !b->tangent) ||
      ((uintptr_t)b->scratch & (kAlign - 1)) != 0 ||
      (b->event_log && b->event_log_capacity <= 0)) {
    free(q);
    return WBRW_ERR_ARG;
  }
  long long n_total = 0;
  double p_max = 0;
  for (int i = 0; i < ninst; ++i) {
    if (q[i].n_init >= (1ll << 32)) { free(q); return WBRW_ERR_ARG; }
    q[i].start = (unsigned long long)n_total;
    n_total += q[i].n_init;
    if (q[i].p_any > p_max) p_max = q[i].p_any;
  }
  const Layout L = layout(config, ninst, b->capacity);
  if (n_total > b->capacity || b->scratch_bytes < L.total) { free(q); return WBRW_ERR_ARG; }

  wbrw_ctx* c = new (std::nothrow) wbrw_ctx();
  if (!c) { free(q); return WBRW_ERR_ARG; }
  c->ih = q;
  c->host_tab = calloc(1, kTabBytes);
  if (!c->host_tab) { free_ctx(c); return WBRW_ERR_ARG; }
  c->ninst = ninst;
  c->cfg = *config;
  c->dim = config->dim;
  if (pot) {
    c->pot = *pot;
  } else {
    c->pot.kind = WBRW_POT_GAUSSIAN;
    c->pot.H = q[0].H;
    c->pot.w = q[0].w;
    c->pot.xc = q[0].xc;
    c->pot.ee = 0;
  }
  c->buf = *b;
  c->stream = (cudaStream_t)cuda_stream;
  c->hm = config->hbar / config->mass;
  c->dtv = config->dt * c->hm;
  // flights short enough that a particle expects at most one candidate
  // interval, so the candidate queue (two entries per particle) holds them
  c->max_chunk = p_max > 0 ? (int)floor(1.0 / p_max) : kMaxChunk;
  if (c->max_chunk > kMaxChunk) c->max_chunk = kMaxChunk;
  if (c->max_chunk < 1) c->max_chunk = 1;
  c->dx = (config->xmax - config->xmin) / (double)config->nx;
  c->dk = (config->kmax - config->kmin) / (double)config->nk;
  c->inv_dx = (double)config->nx / (config->xmax - config->xmin);
  c->inv_dk = (double)config->nk / (config->kmax - config->kmin);
  c->nhi = cells;
  c->nh = c->nhi * ninst;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) !=
          cudaSuccess) {
    free_ctx(c);
    return WBRW_ERR_CUDA;
  }
  char* base = (char*)b->scratch;
  c->cnt = (Counters*)(base + L.counters);
  c->cpid = (unsigned long long*)(base + L.cpid);
  unsigned* counts = (unsigned*)(base + L.seg_counts);
  c->ecnt[0] = counts;
  c->ecnt[1] = counts + (4 + kMaxLevels) * kMaxSeg;
  c->fcnt[0] = counts + kMaxSeg;
  c->fcnt[1] = counts + 2 * kMaxSeg;
  c->dcnt = counts + 3 * kMaxSeg;
  c->rcnt = counts + (3 + kMaxLevels) * kMaxSeg;
  c->cnt_save = (Counters*)(base + L.cnt_save);
  c->fq[0] = base + L.fq0;
  c->fq[1] = base + L.fq1;
  c->qcap = L.qcap;
  c->eq[0] = base + L.eq0;
  c->eq[1] = base + L.eq1;
  c->ecap = L.ecap;
  c->dq[0] = base + L.dq0;
  c->dq[1] = base + L.dq1;
  c->dcap = L.dcap;
  c->rec_cap = L.rec_cap;
  c->passes = 3;
  c->one_launch = 1;
  c->lean = c->cfg.precision == WBRW_FP32 && c->cfg.dim == 2 && ncomp == 0 && !c->buf.event_log;
  c->max_bps = drv(c)->max_bps;
  set_shape(c, c->max_bps);
  c->nz_cell = (uint32_t*)(base + L.nz_cell);
  c->nz_start = (unsigned long long*)(base + L.nz_start);
  c->tile_nz = (uint32_t*)(base + L.tile_nz);
  c->tile_cap = L.tile_cap;
  c->scan_bsum = (unsigned long long*)(base + L.scan_bsum);
  c->scan_bnz = (unsigned int*)(base + L.scan_bnz);
  c->scan_blocks = L.scan_blocks;
  c->tmp_grid = (int*)(base + L.tmp_grid);
  c->tmp_wsum = (long long*)(base + L.tmp_wsum);
  c->obs_density = (double*)(base + L.obs_density);
  c->obs_marg = (double*)(base + L.obs_marg);
  c->obs_col = (long long*)(base + L.obs_col);
  c->obs_scalar = (double*)(base + L.obs_scalar);
  c->rec_cell = (uint32_t*)(base + L.rec_cell);
  c->rec_a = (uint32_t*)(base + L.rec_a);
  c->boot_keep[0] = (int*)(base + L.keep0);
  c->boot_keep[1] = (int*)(base + L.keep1);
  c->boot_res[0] = (unsigned long long*)(base + L.res0);
  c->boot_res[1] = (unsigned long long*)(base + L.res1);
  c->boot_ucnt = (int*)(base + L.ucnt);
  c->boot_guide = (int*)(base + L.guide);
  c->boot_inst = (BootInst*)(base + L.binst);
  c->boot_dpre = (unsigned long long*)(base + L.dpre);
  c->boot_bguide = (int*)(base + L.bguide);
  c->inst_tab = base + L.tabs;
  c->inst_slot = (unsigned long long*)(base + L.tabs + kTabSlotOff);
  c->inst_na = (double*)(base + L.tabs + kTabNaOff);
  c->inst_trans = (double*)(base + L.tabs + kTabTransOff);
  c->cinst = ninst > 1 ? (unsigned*)(base + L.cinst) : nullptr;
  c->obs_red = (long long*)(base + L.obs_red);
  c->ncomp = ncomp;
  c->comp_tab = base + L.tabs + kTabCompOff;
  if (ncomp > 0 && cudaMemcpyAsync(c->comp_tab, comps, (size_t)ncomp * sizeof(Comp),
                                   cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
    free_ctx(c);
    return WBRW_ERR_CUDA;
  }
  c->tangent = config->tangent;
  c->inst_grad = (double*)(base + L.tabs + kTabGradOff);
  c->tinst_slot = (unsigned long long*)(base + L.tabs + kTabTSlotOff);
  if (c->tangent) {
    c->tquantum = tquantum_of(config);
    c->dgrid[0] = (long long*)(base + L.dgrid0);
    c->dgrid[1] = (long long*)(base + L.dgrid1);
    c->tnz_cell = (uint32_t*)(base + L.tnz_cell);
    c->tnz_start = (unsigned long long*)(base + L.tnz_start);
    c->tnz_tau = (double*)(base + L.tnz_tau);
    c->ttile_nz = (uint32_t*)(base + L.ttile_nz);
    if (cudaMemsetAsync(c->dgrid[0], 0, (size_t)c->nh * 8, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->dgrid[1], 0, (size_t)c->nh * 8, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->tinst_slot, 0, (size_t)(kMaxInst + 1) * 8, c->stream) != cudaSuccess) {
      free_ctx(c);
      return WBRW_ERR_CUDA;
    }
  }
  if (c->dim == 4) {
    wbrw_status st = build_tables(c, base, L);
    if (st != WBRW_OK) {
      free_ctx(c);
      return st;
    }
    // the total rate of the three components sets the candidate clock
    c->max_chunk = q[0].p_any > 0 ? (int)floor(1.0 / q[0].p_any) : kMaxChunk;
    if (c->max_chunk > kMaxChunk) c->max_chunk = kMaxChunk;
    if (c->max_chunk < 1) c->max_chunk = 1;
  }
  c->state = ST_PARTICLES;
  c->step = 0;
  c->epoch = 0;
  c->fresh = 0;
  c->failed = 0;
  c->launches = 0;
  c->err[0] = 0;

  cudaError_t e = cudaMemsetAsync(c->cnt, 0, sizeof(Counters), c->stream);
  if (e == cudaSuccess) e = drv(c)->init(c, n_total);
  if (e != cudaSuccess) {
    free_ctx(c);
    return WBRW_ERR_CUDA;
  }
  *out = c;
  return WBRW_OK;
}

}  // namespace

extern "C" {

wbrw_status wbrw_init(const wbrw_config* config, const wbrw_potential* pot,
                      const wbrw_buffers* b, long long n_init, double x0,
                      double sigma_x, double k0, void* cuda_stream,
                      wbrw_ctx** out) {
  if (!out) return WBRW_ERR_ARG;
  *out = nullptr;
  if (!config_ok(config, nullptr, 0) || config->dim != 2) return WBRW_ERR_ARG;
  InstHost* q = (InstHost*)calloc(1, sizeof(InstHost));
  if (!q) return WBRW_ERR_ARG;
  if (!make_instance(config, pot, config->gamma0, x0, sigma_x, k0, n_init, config->n_alpha, q)) {
    free(q);
    return WBRW_ERR_ARG;
  }
  return create(config, nullptr, 1, q, b, cuda_stream, out);
}

wbrw_status wbrw_init_td(const wbrw_config* config, int ncomp, const wbrw_component* comps,
                         const wbrw_buffers* b, long long n_init, double x0, double sigma_x,
                         double k0, void* cuda_stream, wbrw_ctx** out) {
  if (!out) return WBRW_ERR_ARG;
  *out = nullptr;
  if (!config_ok(config, nullptr, 0) || config->dim != 2 || config->tangent) return WBRW_ERR_ARG;
  if (ncomp < 1 || ncomp > kMaxComp || !comps) return WBRW_ERR_ARG;
  if (!(sigma_x > 0) || !isfinite(sigma_x) || !isfinite(x0) || !isfinite(k0) || n_init < 0)
    return WBRW_ERR_ARG;
  Comp tab[kMaxComp];
  memset(tab, 0, sizeof(tab));
  double G = 0.0;
  for (int m = 0; m < ncomp; ++m) {
    const wbrw_component& v = comps[m];
    if (!(v.w > 0) || !isfinite(v.w) || !isfinite(v.a) || !isfinite(v.b) || !isfinite(v.omega) ||
        !isfinite(v.phase) || !isfinite(v.xc))
      return WBRW_ERR_ARG;
    tab[m].a = v.a;
    tab[m].b = v.b;
    tab[m].om = v.omega;
    tab[m].ph = v.phase;
    tab[m].sig_k = 1.0 / (2.0 * v.w);
    tab[m].xc = v.xc;
    tab[m].gam = (fabs(v.a) + fabs(v.b)) / config->hbar;
    tab[m].hg = config->hbar * tab[m].gam;
    G += tab[m].gam;
  }
  InstHost* q = (InstHost*)calloc(1, sizeof(InstHost));
  if (!q) return WBRW_ERR_ARG;
  q->w = 1.0;
  q->x0 = x0;
  q->sx = sigma_x;
  q->k0 = k0;
  q->n_init = n_init;
  q->n_alpha = config->n_alpha;
  q->gamma0 = G > 0.0 ? G : 1.0;  // no potential: no pair is ever made
  q->cacc = 1.0;
  q->p_any = -expm1(-q->gamma0 * config->dt);
  return create(config, nullptr, 1, q, b, cuda_stream, out, ncomp, tab);
}

wbrw_status wbrw_init4d(const wbrw_config* config, const wbrw_potential* pot,
                        const wbrw_buffers* b, long long n_init, const double x0[2],
                        double sigma_x, const double k0[2], void* cuda_stream, wbrw_ctx** out) {
  if (!out) return WBRW_ERR_ARG;
  *out = nullptr;
  if (!config_ok(config, nullptr, 0) || config->dim != 4 || !x0 || !k0) return WBRW_ERR_ARG;
  if (!pot || pot->kind != WBRW_POT_SOFT_COULOMB_2E || !(pot->w > 0) || !isfinite(pot->w) ||
      !isfinite(pot->H) || !isfinite(pot->xc) || !isfinite(pot->ee))
    return WBRW_ERR_ARG;
  if (!(sigma_x > 0) || !isfinite(sigma_x) || n_init < 0 || !isfinite(x0[0]) ||
      !isfinite(x0[1]) || !isfinite(k0[0]) || !isfinite(k0[1]))
    return WBRW_ERR_ARG;
  InstHost* q = (InstHost*)calloc(1, sizeof(InstHost));
  if (!q) return WBRW_ERR_ARG;
  q->H = pot->H;
  q->w = pot->w;
  q->xc = pot->xc;
  q->x0 = x0[0];
  q->x0b = x0[1];
  q->sx = sigma_x;
  q->k0 = k0[0];
  q->k0b = k0[1];
  q->n_init = n_init;
  q->n_alpha = config->n_alpha;
  q->gamma0 = 1.0;  // set with the tables
  q->p_any = 0.0;
  return create(config, pot, 1, q, b, cuda_stream, out);
}

wbrw_status wbrw_batch_init(const wbrw_config* config, int ninst, const wbrw_instance* inst,
                            const wbrw_buffers* b, void* cuda_stream, wbrw_ctx** out) {
  if (!out) return WBRW_ERR_ARG;
  *out = nullptr;
  if (ninst < 1 || !inst || !config_ok(config, nullptr, 0, ninst) || config->dim != 2)
    return WBRW_ERR_ARG;
  InstHost* q = (InstHost*)calloc((size_t)ninst, sizeof(InstHost));
  if (!q) return WBRW_ERR_ARG;
  for (int i = 0; i < ninst; ++i) {
    const wbrw_instance& v = inst[i];
    if (!make_instance(config, &v.pot, v.gamma0, v.x0, v.sigma_x, v.k0, v.n_init, v.n_alpha,
                       &q[i])) {
      free(q);
      return WBRW_ERR_ARG;
    }
  }
  return create(config, nullptr, ninst, q, b, cuda_stream, out);
}

wbrw_status wbrw_step(wbrw_ctx* c, int nsteps) {
  if (!c) return WBRW_ERR_ARG;
  if (c->failed) return WBRW_ERR_STATE;
  if (nsteps < 0) return seterr(c, WBRW_ERR_ARG, "nsteps must be >= 0");
  return step_impl(c, nsteps);
}

wbrw_status wbrw_annihilate(wbrw_ctx* c) {
  if (!c) return WBRW_ERR_ARG;
  if (c->failed) return WBRW_ERR_STATE;
  if (c->fresh) return WBRW_OK;
  wbrw_status st = ensure_particles(c);
  if (st != WBRW_OK) return st;
  c->epoch += 1;
  st = resample_from_arrays(c);
  if (st != WBRW_OK) return st;
  c->state = ST_HISTOGRAM;
  c->fresh = 1;
  return WBRW_OK;
}

wbrw_status wbrw_run(wbrw_ctx* c, int nsteps) {
  if (!c) return WBRW_ERR_ARG;
  if (c->failed) return WBRW_ERR_STATE;
  if (nsteps < 0) return seterr(c, WBRW_ERR_ARG, "nsteps must be >= 0");
  const int T = c->cfg.resample_every;
  if (T <= 0) return step_impl(c, nsteps);
  while (nsteps > 0) {
    const int to_boundary = T - (int)(c->step % T);
    if (nsteps < to_boundary || to_boundary > c->max_chunk) {
      // no resampling inside this piece: plain steps into the arrays
      int ch = nsteps < to_boundary ? nsteps : to_boundary - c->max_chunk;
      if (ch > c->max_chunk) ch = c->max_chunk;
      wbrw_status st = step_impl(c, ch);
      if (st != WBRW_OK) return st;
      nsteps -= ch;
      continue;
    }
    // one fused period: (regenerate) + fly to the boundary + histogram
    const int src = c->state == ST_HISTOGRAM ? SRC_REGEN : SRC_ARRAY;
    const int l0 = (int)c->step, L = l0 + to_boundary;
    const long long regen_epoch = c->epoch;
    wbrw_status st;
    if (c->graph_on && src == SRC_REGEN)
      st = graph_period(c, to_boundary);
    else
      st = enqueue_period(c, src, l0, L, regen_epoch);
    if (st != WBRW_OK) return st;
    c->epoch = regen_epoch + 1;  // the histogram this period produced
    c->step = L;
    c->state = ST_HISTOGRAM;
    c->fresh = 1;
    nsteps -= to_boundary;
  }
  return WBRW_OK;
}

wbrw_status wbrw_instance_density(wbrw_ctx* c, int inst, double* density_host,
                                  double* marginal_x_host, double* transmission,
                                  long long* live_particles) {
  if (!c) return WBRW_ERR_ARG;
  if (c->failed) return WBRW_ERR_STATE;
  if (inst < 0 || inst >= c->ninst) return seterr(c, WBRW_ERR_ARG, "no instance %d", inst);
  wbrw_status st;
  if (c->state == ST_HISTOGRAM) {
    WBRW_TRY(c, launch_observables(c, inst, c->buf.grid, nullptr), "observables");
  } else if (c->cfg.strategy == WBRW_SP1_PAIR) {
    WBRW_TRY(c, launch_zero(c, c->tmp_grid, (size_t)c->nh * 4), "zero");
    WBRW_TRY(c, drv(c)->bin(c, DST_BIN1, c->tmp_grid, 0), "bin");
    WBRW_TRY(c, launch_observables(c, inst, c->tmp_grid, nullptr), "observables");
  } else {
    WBRW_TRY(c, launch_zero(c, c->tmp_wsum, (size_t)c->nh * 8), "zero");
    WBRW_TRY(c, drv(c)->bin(c, DST_WSUM, c->tmp_grid, 0), "bin");
    WBRW_TRY(c, launch_observables(c, inst, nullptr, c->tmp_wsum), "observables");
  }
  if (density_host)
    WBRW_TRY(c, cudaMemcpyAsync(density_host, c->obs_density,
                                (size_t)c->cfg.nx * c->cfg.nk * 8,
                                cudaMemcpyDeviceToHost, c->stream), "copy density");
  if (marginal_x_host)
    WBRW_TRY(c, cudaMemcpyAsync(marginal_x_host, c->obs_marg, (size_t)c->cfg.nx * 8,
                                cudaMemcpyDeviceToHost, c->stream), "copy marginal");
  double T = 0;
  unsigned long long live = 0;
  WBRW_TRY(c, cudaMemcpyAsync(&T, c->obs_scalar, 8, cudaMemcpyDeviceToHost, c->stream), "copy");
  if (c->ninst == 1) {
    WBRW_TRY(c, cudaMemcpyAsync(&live, c->state == ST_HISTOGRAM ? &c->cnt->regen_total
                                                                : &c->cnt->n,
                                8, cudaMemcpyDeviceToHost, c->stream), "copy");
  } else if (c->state == ST_HISTOGRAM) {
    unsigned long long se[2];
    WBRW_TRY(c, cudaMemcpyAsync(se, c->inst_slot + inst, 16, cudaMemcpyDeviceToHost, c->stream),
             "copy");
    WBRW_TRY(c, cudaStreamSynchronize(c->stream), "synchronise");
    live = se[1] - se[0];
  } else {
    unsigned long long* d = (unsigned long long*)(c->obs_scalar + 1);
    WBRW_TRY(c, launch_zero(c, d, 8), "zero");
    WBRW_TRY(c, launch_live_instance(c, inst, d), "count");
    WBRW_TRY(c, cudaMemcpyAsync(&live, d, 8, cudaMemcpyDeviceToHost, c->stream), "copy");
  }
  st = device_status(c);
  if (st != WBRW_OK) return st;
  if (transmission) *transmission = T;
  if (live_particles) *live_particles = (long long)live;
  return WBRW_OK;
}

wbrw_status wbrw_density(wbrw_ctx* c, double* density_host, double* marginal_x_host,
                         double* transmission, long long* live_particles) {
  return wbrw_instance_density(c, 0, density_host, marginal_x_host, transmission,
                               live_particles);
}

wbrw_status wbrw_transmissions(wbrw_ctx* c, double* out_host) {
  if (!c || !out_host) return WBRW_ERR_ARG;
  if (c->failed) return WBRW_ERR_STATE;
  if (c->state != ST_HISTOGRAM)
    return seterr(c, WBRW_ERR_STATE, "transmissions need a resampling first");
  if (c->dim == 4) {
    WBRW_TRY(c, launch_observables(c, 0, c->buf.grid, nullptr), "observables");
    WBRW_TRY(c, cudaMemcpyAsync(out_host, c->obs_scalar, 8, cudaMemcpyDeviceToHost, c->stream),
             "copy");
    return device_status(c);
  }
  WBRW_TRY(c, launch_transmissions(c, c->buf.grid, c->inst_trans), "transmissions");
  WBRW_TRY(c, cudaMemcpyAsync(out_host, c->inst_trans, (size_t)c->ninst * 8,
                              cudaMemcpyDeviceToHost, c->stream), "copy");
  return device_status(c);
}

wbrw_status wbrw_transmission_gradients(wbrw_ctx* c, double* out_host) {
  if (!c || !out_host) return WBRW_ERR_ARG;
  if (c->failed) return WBRW_ERR_STATE;
  if (!c->tangent) return seterr(c, WBRW_ERR_STATE, "the context carries no tangents");
  if (c->state != ST_HISTOGRAM)
    return seterr(c, WBRW_ERR_STATE, "gradients need a resampling first");
  WBRW_TRY(c, launch_transmission_gradients(c), "gradients");
  WBRW_TRY(c, cudaMemcpyAsync(out_host, c->inst_grad, (size_t)c->ninst * 16,
                              cudaMemcpyDeviceToHost, c->stream), "copy");
  return device_status(c);
}

wbrw_status wbrw_particle_instances(wbrw_ctx* c, unsigned int* inst_dev) {
  if (!c || !inst_dev) return WBRW_ERR_ARG;
  if (c->failed) return WBRW_ERR_STATE;
  if (c->state != ST_PARTICLES)
    return seterr(c, WBRW_ERR_STATE, "particles are not materialised");
  WBRW_TRY(c, drv(c)->pids(c, nullptr, inst_dev), "instances");
  return device_status(c);
}

wbrw_status wbrw_particles(wbrw_ctx* c, long long* n_host, unsigned long long* pid_dev) {
  if (!c) return WBRW_ERR_ARG;
  if (c->failed) return WBRW_ERR_STATE;
  wbrw_status st = ensure_particles(c);
  if (st != WBRW_OK) return st;
  if (pid_dev) WBRW_TRY(c, drv(c)->pids(c, pid_dev, nullptr), "ids");
  unsigned long long n = 0;
  WBRW_TRY(c, cudaMemcpyAsync(&n, &c->cnt->n, 8, cudaMemcpyDeviceToHost, c->stream), "copy");
  st = device_status(c);
  if (st != WBRW_OK) return st;
  if (n_host) *n_host = (long long)n;
  return WBRW_OK;
}

wbrw_status wbrw_counters(wbrw_ctx* c, long long* out) {
  if (!c || !out) return WBRW_ERR_ARG;
  Counters h;
  WBRW_TRY(c, cudaMemcpyAsync(&h, c->cnt, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream),
           "copy counters");
  WBRW_TRY(c, cudaStreamSynchronize(c->stream), "synchronise");
  for (int i = 0; i < WBRW_C_COUNT; ++i) out[i] = 0;
  out[WBRW_C_LIVE] = (long long)(c->state == ST_HISTOGRAM ? h.regen_total : h.n);
  out[WBRW_C_EVENTS] = (long long)h.ledger[LG_EVENTS];
  out[WBRW_C_KILL_PLUS] = (long long)h.ledger[LG_KILL_P];
  out[WBRW_C_KILL_MINUS] = (long long)h.ledger[LG_KILL_M];
  out[WBRW_C_OUT_PLUS] = (long long)h.ledger[LG_OUT_P];
  out[WBRW_C_OUT_MINUS] = (long long)h.ledger[LG_OUT_M];
  out[WBRW_C_PARTICLE_STEPS] = (long long)(h.ledger[LG_PSTEPS] + h.ledger[LG_PSTEPS0]);
  out[WBRW_C_PARTICLE_STEPS_FIRST] = (long long)h.ledger[LG_PSTEPS0];
  out[WBRW_C_CANDIDATES] = (long long)h.ledger[LG_CAND];
  out[WBRW_C_FIRST_PAIRS] = (long long)h.ledger[LG_PAIRS0];
  out[WBRW_C_LOG_LEN] = (long long)h.log_len;
  out[WBRW_C_STEP] = c->step;
  out[WBRW_C_EPOCH] = c->epoch;
  out[WBRW_C_LAUNCHES] = c->launches;
  out[WBRW_C_BOOT_NPLUS] = (long long)h.boot_n[0];
  out[WBRW_C_BOOT_NMINUS] = (long long)h.boot_n[1];
  out[WBRW_C_BOOT_NRPLUS] = (long long)h.boot_nr[0];
  out[WBRW_C_BOOT_NRMINUS] = (long long)h.boot_nr[1];
  out[WBRW_C_BOOT_WPLUS] = (long long)h.boot_w[0];
  out[WBRW_C_BOOT_WMINUS] = (long long)h.boot_w[1];
  out[WBRW_C_NONZERO_CELLS] = (long long)h.nz_count;
  out[WBRW_C_ERROR] = h.err;
  if (h.err) return device_status(c);
  return WBRW_OK;
}

wbrw_status wbrw_sync_status(wbrw_ctx* c) {
  if (!c) return WBRW_ERR_ARG;
  if (c->failed) return WBRW_ERR_STATE;
  return device_status(c);
}

const char* wbrw_last_error(const wbrw_ctx* c) {
  if (!c) return "NULL context";
  return c->err;
}

wbrw_status wbrw_checkpoint(wbrw_ctx* c, int* grid_out, long long* step, long long* epoch) {
  if (!c || !grid_out) return WBRW_ERR_ARG;
  if (c->failed) return WBRW_ERR_STATE;
  if (!c->fresh) return seterr(c, WBRW_ERR_STATE, "checkpoint needs a resampling first");
  WBRW_TRY(c, cudaMemcpyAsync(grid_out, c->buf.grid, (size_t)c->nh * 4, cudaMemcpyDefault,
                              c->stream), "copy grid");
  wbrw_status st = device_status(c);
  if (st != WBRW_OK) return st;
  if (step) *step = c->step;
  if (epoch) *epoch = c->epoch;
  return WBRW_OK;
}

wbrw_status wbrw_restore(wbrw_ctx* c, const int* grid, long long step, long long epoch) {
  if (!c || !grid) return WBRW_ERR_ARG;
  if (c->failed) return WBRW_ERR_STATE;
  if (step < 0 || step >= (1ll << 31) || epoch < 0 || epoch >= (1ll << 23))
    return seterr(c, WBRW_ERR_ARG, "step or epoch out of range");
  WBRW_TRY(c, cudaMemcpyAsync(c->buf.grid, grid, (size_t)c->nh * 4, cudaMemcpyDefault,
                              c->stream), "copy grid");
  WBRW_TRY(c, launch_scan_cells(c, c->buf.grid), "scan");
  if (c->tangent) {
    WBRW_TRY(c, zero_tangent(c), "zero tangent");
    WBRW_TRY(c, launch_scan_tangent(c), "tangent plan");
  }
  c->step = step;
  c->epoch = epoch;
  c->state = ST_HISTOGRAM;
  c->fresh = 1;
  c->dev_period_ok = 0;
  return WBRW_OK;
}

// The side stream and fork/join events of the profiling records.
static wbrw_status ensure_side(wbrw_ctx* c) {
  if (c->prof_side_created) return WBRW_OK;
  WBRW_TRY(c, cudaEventCreateWithFlags(&c->prof_fork, cudaEventDisableTiming), "create events");
  WBRW_TRY(c, cudaEventCreateWithFlags(&c->prof_join, cudaEventDisableTiming), "create events");
  WBRW_TRY(c, cudaStreamCreateWithFlags(&c->prof_side, cudaStreamNonBlocking), "create stream");
  c->prof_side_created = 1;
  return WBRW_OK;
}

wbrw_status wbrw_graph(wbrw_ctx* c, int enable) {
  if (!c) return WBRW_ERR_ARG;
  if (c->failed) return WBRW_ERR_STATE;
  if (enable && !c->gev_created) {
    for (int i = 0; i < 2 + 2 * kProfRounds; ++i)
      WBRW_TRY(c, cudaEventCreateWithFlags(&c->gev[i], cudaEventDefault), "create events");
    c->gev_created = 1;
  }
  if (enable) {
    const wbrw_status st = ensure_side(c);
    if (st != WBRW_OK) return st;
  }
  if (enable) {
    cudaStreamCaptureStatus cs;
    WBRW_TRY(c, cudaStreamIsCapturing(c->stream, &cs), "stream");
    if (c->stream == nullptr || c->stream == cudaStreamLegacy ||
        c->stream == cudaStreamPerThread || cs != cudaStreamCaptureStatusNone)
      return seterr(c, WBRW_ERR_ARG, "graph capture needs a created, non-capturing stream");
  } else {
    WBRW_TRY(c, cudaStreamSynchronize(c->stream), "synchronise");
    drop_graphs(c);
  }
  c->graph_on = enable ? 1 : 0;
  return WBRW_OK;
}

wbrw_status wbrw_get_tuning(wbrw_ctx* c, wbrw_tuning* out) {
  if (!c || !out) return WBRW_ERR_ARG;
  out->blocks_per_sm = c->bps;
  out->event_passes = c->passes;
  return WBRW_OK;
}

wbrw_status wbrw_one_launch_periods(wbrw_ctx* c, int enable) {
  if (!c) return WBRW_ERR_ARG;
  if (c->failed) return WBRW_ERR_STATE;
  if ((enable ? 1 : 0) != c->one_launch) {
    WBRW_TRY(c, cudaStreamSynchronize(c->stream), "synchronise");
    drop_graphs(c);
    c->one_launch = enable ? 1 : 0;
  }
  return WBRW_OK;
}

wbrw_status wbrw_set_tuning(wbrw_ctx* c, const wbrw_tuning* t) {
  if (!c || !t) return WBRW_ERR_ARG;
  if (c->failed) return WBRW_ERR_STATE;
  if (t->blocks_per_sm < 1 || t->blocks_per_sm > c->max_bps || t->event_passes < 0 ||
      t->event_passes > kMaxPasses)
    return seterr(c, WBRW_ERR_ARG, "tuning out of range");
  if (t->blocks_per_sm != c->bps || t->event_passes != c->passes) {
    WBRW_TRY(c, cudaStreamSynchronize(c->stream), "synchronise");
    drop_graphs(c);
    set_shape(c, t->blocks_per_sm);
    c->passes = t->event_passes;
  }
  return WBRW_OK;
}

wbrw_status wbrw_autotune(wbrw_ctx* c, int trials, wbrw_tuning* best, double* ms_table) {
  if (!c || trials < 1) return WBRW_ERR_ARG;
  if (c->failed) return WBRW_ERR_STATE;
  if (!c->fresh || c->state != ST_HISTOGRAM || c->cfg.resample_every <= 0)
    return seterr(c, WBRW_ERR_STATE, "autotune needs the state right after a resampling");
  if (c->tangent)
    return seterr(c, WBRW_ERR_STATE, "autotune a context without tangents (same shapes)");
  const int T = c->cfg.resample_every;
  const int len = T - (int)(c->step % T);
  if (len > c->max_chunk)
    return seterr(c, WBRW_ERR_STATE, "the period is longer than one flight");
  // what the trials disturb, to be put back
  const long long step0 = c->step, epoch0 = c->epoch, launches0 = c->launches;
  const int prof0 = c->prof_on, graph0 = c->graph_on, bps0 = c->bps, passes0 = c->passes;
  void* log0 = c->buf.event_log;
  WBRW_TRY(c, cudaStreamSynchronize(c->stream), "synchronise");
  drop_graphs(c);
  c->prof_on = 0;
  c->graph_on = 0;
  c->buf.event_log = nullptr;
  WBRW_TRY(c, cudaMemcpyAsync(c->cnt_save, c->cnt, sizeof(Counters), cudaMemcpyDeviceToDevice,
                              c->stream), "save counters");
  WBRW_TRY(c, cudaMemcpyAsync(c->tmp_grid, c->buf.grid, (size_t)c->nh * 4,
                              cudaMemcpyDeviceToDevice, c->stream), "save grid");
  cudaEvent_t ev[2];
  WBRW_TRY(c, cudaEventCreate(&ev[0]), "event");
  if (cudaEventCreate(&ev[1]) != cudaSuccess) {
    cudaEventDestroy(ev[0]);
    return seterr(c, WBRW_ERR_CUDA, "event");
  }
  auto put_back = [&]() -> wbrw_status {
    WBRW_TRY(c, cudaMemcpyAsync(c->buf.grid, c->tmp_grid, (size_t)c->nh * 4,
                                cudaMemcpyDeviceToDevice, c->stream), "restore grid");
    WBRW_TRY(c, cudaMemcpyAsync(c->cnt, c->cnt_save, sizeof(Counters),
                                cudaMemcpyDeviceToDevice, c->stream), "restore counters");
    WBRW_TRY(c, launch_scan_cells(c, c->buf.grid), "scan");
    c->step = step0;
    c->epoch = epoch0;
    c->state = ST_HISTOGRAM;
    c->fresh = 1;
    c->dev_period_ok = 0;
    return WBRW_OK;
  };
  double best_ms = -1;
  int best_b = bps0, best_p = passes0;
  wbrw_status st = WBRW_OK;
  if (ms_table)  // shapes beyond what this context's kernels are built for
    for (int i = 0; i < kMaxBlocksPerSm * (kMaxPasses + 1); ++i) ms_table[i] = -1.0;
  // kernels that finish deferred segments inside the event kernel: there
  // event_passes changes nothing, and only 0 is timed
  const int max_pz = drv(c)->inline_drain ? 0 : kMaxPasses;
  for (int b = 1; b <= c->max_bps && st == WBRW_OK; ++b) {
    for (int pz = 0; pz <= max_pz && st == WBRW_OK; ++pz) {
      set_shape(c, b);
      c->passes = pz;
      double t_min = -1;
      for (int t = 0; t < trials && st == WBRW_OK; ++t) {
        if ((st = put_back()) != WBRW_OK) break;
        if ((st = cuda_check(c, cudaEventRecord(ev[0], c->stream), "record")) != WBRW_OK) break;
        if ((st = enqueue_period(c, SRC_REGEN, (int)step0, (int)step0 + len, epoch0)) != WBRW_OK)
          break;
        if ((st = cuda_check(c, cudaEventRecord(ev[1], c->stream), "record")) != WBRW_OK) break;
        int err = 0;
        if ((st = cuda_check(c, cudaMemcpyAsync(&err, &c->cnt->err, sizeof(int),
                                                cudaMemcpyDeviceToHost, c->stream),
                             "read error word")) != WBRW_OK)
          break;
        if ((st = cuda_check(c, cudaStreamSynchronize(c->stream), "synchronise")) != WBRW_OK)
          break;
        float ms = 0;
        if ((st = cuda_check(c, cudaEventElapsedTime(&ms, ev[0], ev[1]), "elapsed")) != WBRW_OK)
          break;
        if (err) { t_min = -1; break; }  // a capacity limit under this shape
        if (t_min < 0 || ms < t_min) t_min = ms;
      }
      if (ms_table) ms_table[(b - 1) * (kMaxPasses + 1) + pz] = t_min;
      if (t_min >= 0 && (best_ms < 0 || t_min < best_ms)) {
        best_ms = t_min;
        best_b = b;
        best_p = pz;
      }
    }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (st != WBRW_OK) return st;
  set_shape(c, best_b);
  c->passes = best_p;
  st = put_back();
  if (st != WBRW_OK) return st;
  c->launches = launches0;
  c->prof_on = prof0;
  c->graph_on = graph0;
  c->buf.event_log = log0;
  if (best) {
    best->blocks_per_sm = best_b;
    best->event_passes = best_p;
  }
  return device_status(c);
}

wbrw_status wbrw_profile(wbrw_ctx* c, int enable) {
  if (!c) return WBRW_ERR_ARG;
  if (enable) {
    const wbrw_status st = ensure_side(c);
    if (st != WBRW_OK) return st;
  }
  if (enable && !c->prof_created) {
    for (int i = 0; i < 2 * kProfLaunches; ++i) {
      WBRW_TRY(c, cudaEventCreate(&c->prof_ev[i]), "create events");
      WBRW_TRY(c, cudaEventCreate(&c->prof_evk[i]), "create events");
    }
    c->prof_created = 1;
  }
  c->prof_on = enable ? 1 : 0;
  c->prof_n = 0;
  c->prof_nk = 0;
  return WBRW_OK;
}

wbrw_status wbrw_profile_read(wbrw_ctx* c, double* total_ms, long long* launches) {
  if (!c) return WBRW_ERR_ARG;
  WBRW_TRY(c, cudaStreamSynchronize(c->stream), "synchronise");
  if (c->prof_side_created)
    WBRW_TRY(c, cudaStreamSynchronize(c->prof_side), "synchronise");
  double t = 0;
  for (int i = 0; i < c->prof_n; ++i) {
    float ms = 0;
    WBRW_TRY(c, cudaEventElapsedTime(&ms, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]), "elapsed");
    t += ms;
  }
  if (total_ms) *total_ms = t;
  if (launches) *launches = c->prof_n;
  c->prof_n = 0;
  return WBRW_OK;
}

wbrw_status wbrw_profile_read_events(wbrw_ctx* c, double* total_ms, long long* launches) {
  if (!c) return WBRW_ERR_ARG;
  WBRW_TRY(c, cudaStreamSynchronize(c->stream), "synchronise");
  if (c->prof_side_created)
    WBRW_TRY(c, cudaStreamSynchronize(c->prof_side), "synchronise");
  double t = 0;
  for (int i = 0; i < c->prof_nk; ++i) {
    float ms = 0;
    WBRW_TRY(c, cudaEventElapsedTime(&ms, c->prof_evk[2 * i], c->prof_evk[2 * i + 1]),
             "elapsed");
    t += ms;
  }
  if (total_ms) *total_ms = t;
  if (launches) *launches = c->prof_nk;
  c->prof_nk = 0;
  return WBRW_OK;
}

void wbrw_destroy(wbrw_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  if (c->gev_created)
    for (int i = 0; i < 2 + 2 * kProfRounds; ++i) cudaEventDestroy(c->gev[i]);
  if (c->prof_side_created) {
    cudaStreamSynchronize(c->prof_side);
    cudaEventDestroy(c->prof_fork);
    cudaEventDestroy(c->prof_join);
    cudaStreamDestroy(c->prof_side);
  }
  if (c->prof_created)
    for (int i = 0; i < 2 * kProfLaunches; ++i) {
      cudaEventDestroy(c->prof_ev[i]);
      cudaEventDestroy(c->prof_evk[i]);
    }
  free_ctx(c);
}

}  // extern "C"
