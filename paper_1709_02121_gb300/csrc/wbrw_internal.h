// wbrw_internal.h -- host-side context shared by the C-ABI translation unit
// and the per-precision kernel drivers.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "wbrw.h"

namespace wbrw {

constexpr int kBlock = 256;      // threads per block of every particle kernel
constexpr int kMaxChunk = 32;    // steps fused in one flight (bits of a mask)
constexpr int kScanItems = 8;    // cells per thread in the cell scans
constexpr int kScanTile = kBlock * kScanItems;
constexpr int kTabGuideBits = 8;  // 4D kick rows (FP32): guide table of 2^8 buckets per row
constexpr int kTabGuide = 1 << kTabGuideBits;
constexpr int kGuideBits = 16;  // sp2 draws: guide table of 2^16 buckets per side
constexpr int kGuide = 1 << kGuideBits;
constexpr int kGuideBitsB = 14;  // sp2 draws of a batch: 2^14 buckets per instance and side
constexpr int kGuideB = 1 << kGuideBitsB;
constexpr int kMaxSeg = 8192;    // most queue segments (one per producer warp)
constexpr int kMaxBlocksPerSm = WBRW_TUNE_BLOCKS_PER_SM_MAX;  // the largest launch bound of the
                                                             // queue kernels (see max_blocks)
// Deferred-segment levels of the event kernels: level 1 is fed by the first
// event of each candidate interval, levels 1..passes are finished one event
// per lockstep pass, level passes + 1 by the recursive drain.
constexpr int kMaxPasses = WBRW_TUNE_PASSES_MAX;
constexpr int kMaxLevels = kMaxPasses + 2;
constexpr int kMaxInst = WBRW_MAX_INSTANCES;  // instances of a batch (8 id bits)
constexpr int kInstBytes = 128;               // one per-instance record on the device
constexpr size_t kInstTabBytes = (size_t)kMaxInst * kInstBytes;
// device tables: physics records, initial-sampling records, first slots,
// N_alpha (double) and the transmissions read-out, in this order; the host
// stages all but the last
constexpr size_t kTabSlotOff = 2 * kInstTabBytes;
constexpr size_t kTabNaOff = kTabSlotOff + (size_t)(kMaxInst + 1) * 8;
constexpr size_t kTabTransOff = kTabNaOff + (size_t)kMaxInst * 8;
// tangent mode: the first slot of each instance's tangent particles, and the
// read-out of (dT/dH, dT/dw) per instance
constexpr size_t kTabTSlotOff = kTabTransOff + (size_t)kMaxInst * 8;
constexpr size_t kTabGradOff = kTabTSlotOff + (size_t)(kMaxInst + 1) * 8;
constexpr size_t kTabCompOff = kTabGradOff + (size_t)kMaxInst * 16;
constexpr int kMaxComp = WBRW_MAX_COMPONENTS;  // components of a time-dependent V
constexpr size_t kTabBytes = kTabCompOff + (size_t)kMaxComp * 64;

// SRC_TREGEN: the tangent mode's sign-0 particles regenerated from the
// tangent histogram (a second plan).
enum Src { SRC_ARRAY = 0, SRC_REGEN = 1, SRC_QUEUE = 2, SRC_TREGEN = 3 };
enum Dst { DST_ARRAY = 0, DST_BIN1 = 1, DST_BIN2 = 2, DST_WSUM = 3 };

// device error bits (Counters::err)
enum : int {
  ERR_CAP_PARTICLES = 1,
  ERR_CAP_QUEUE = 2,
  ERR_CAP_EQUEUE = 4,
  ERR_NESTING = 8,
  ERR_CAP_RECORDS = 16,
  ERR_NUMERIC = 32,  // a non-finite position or wavevector reached binning
};

// ledger slots (Counters::ledger)
// LG_CAND: candidate intervals whose first event the event kernel performed;
// LG_PAIRS0: those of them that emitted a pair.
enum {
  LG_EVENTS = 0, LG_KILL_P, LG_KILL_M, LG_OUT_P, LG_OUT_M, LG_PSTEPS, LG_PSTEPS0, LG_CAND,
  LG_PAIRS0, LG_N = 10
};

// Device-resident counters: every count the host would otherwise need lives
// here, so no launch waits for the host.
struct Counters {
  unsigned long long n;            // particles in the arrays
  unsigned long long n_src;        // snapshot of n at the start of a chunk
  unsigned long long n_base;       // slots < n_base have pid = base_pid + slot
  unsigned long long base_pid;
  unsigned long long nz_count;     // nonzero cells of the last histogram
  unsigned long long regen_total;  // particles implied by the histogram
  unsigned long long log_len;
  unsigned long long ledger[LG_N];
  unsigned long long boot_n[2], boot_w[2], boot_keep[2], boot_nr[2];
  unsigned long long boot_R[2];    // total residual (Q0.32) per side
  long long obs_total;             // observables: transmission numerator
  unsigned long long per_regen_base;  // the chunk's regeneration id base (epoch << 40)
  unsigned long long tan_total;       // tangent particles implied by the tangent histogram
  unsigned long long tan_nz;          // cells carrying tangent weight
  int per_l0;                         // the chunk's first interval
  int err;
  int pad[2];
};

// The signed bootstrap of a batch (sp2, Alg. 2 per instance and side): one
// record per instance in device memory.  The counts and weight sums come
// from the instance's records and unit-weight counts, the shares from them,
// the residual prefix is taken over the cells of all instances (base: its
// value before the instance's first cell).
struct BootInst {
  unsigned long long n[2], w[2];     // N^s and W^s (Q1.31)
  unsigned long long keep[2];        // sum of floor(q_i)
  unsigned long long base[2], R[2];  // residual prefix before the instance's cells; its total
  unsigned long long nr[2];          // the N_r^s residual draws
  double ratio[2], amp[2];           // N^s / W^s; (W^s 2^-31) / N^s
  unsigned long long mx[2];          // floor(N^s 2^64 / W^s) where the fixed-point shares apply
  int fx[2];
  int kf_unit[2];                    // the share of a unit weight: integer part
  unsigned long long res_unit[2];    //   and Q0.32 residual
};

// Rounds of a captured period whose event kernel a graph replay can time,
// and launches each profiling buffer keeps.
constexpr int kProfRounds = 64;
constexpr int kProfLaunches = 4096;

// A resampling period of wbrw_run captured into a CUDA graph (sp1, source =
// the regeneration of the previous histogram), keyed by its length.  The
// event records of the profiling are captured only while profiling is on
// (each costs a few microseconds per replay); a replay in the other state
// captures the period again.
struct PeriodGraph {
  int len;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  cudaGraphNode_t ev_begin, ev_end;  // event records around the first wave
  // event records around the event kernel of round r < kProfRounds
  cudaGraphNode_t evk_begin[kProfRounds], evk_end[kProfRounds];
  int nevk;                          // rounds with both records
  int evk_live;                      // they point at profiling events
  int prof;                          // captured while profiling: the records exist
  long long launches;                // kernels in the graph
};
constexpr int kMaxGraphs = 4;

// One Gaussian component of a time-dependent potential, as the kernels read
// it: V_m(x, t) = (a + b cos(om t + ph)) exp(-(x - xc)^2/(2 w^2)),
// sig_k = 1/(2w), gam = (|a| + |b|)/hbar (its majorant rate), hg = hbar gam.
struct Comp {
  double a, b, om, ph, sig_k, xc, gam, hg;
};

// One instance of a batch, host FP64 (Sec. 4.2 / Remark 3 / Sec. 3.2).
struct InstHost {
  double H, w, xc;             // potential
  double C, sig_k, gamma0, cacc, p_any;
  double x0, sx, k0;           // initial wavepacket
  double x0b, k0b;             // 4D model: the second electron's packet
  long long n_init, n_alpha;
  unsigned long long start;    // first slot of its initial particles
};

struct Ctx {
  wbrw_config cfg;
  wbrw_potential pot;
  wbrw_buffers buf;
  cudaStream_t stream;
  int device;
  int num_sms;
  // constants (Sec. 4.2 / Remark 3 / Sec. 3.2), host FP64; per instance in ih
  double hm, dtv, dx, dk, inv_dx, inv_dk;
  int ninst;          // instances (1 for wbrw_init)
  InstHost* ih;       // ninst records (host)
  void* host_tab;     // staging copy of the device tables (kTabBytes)
  long long nhi;      // cells per instance
  long long nh;       // cells of all instances (ninst nhi)
  void* inst_tab;     // device tables (kTabBytes, in the scratch)
  unsigned long long* inst_slot;  // first slot of each instance's base particles (+ total)
  unsigned* cinst;    // instance of each appended offspring (batches only)
  double* inst_na;    // N_alpha of each instance (device)
  double* inst_trans; // transmissions read-out (device)
  // 4D model: kernel tables in the scratch (type 0: one-body, 1: interaction)
  int dim;            // 2 or 4
  int tab_ny, tab_nkap;
  double tab_Y[2], tab_dy[2], tab_inv_dy[2], tab_gam[2], tab_K, tab_dkap;
  double* tab_A;                  // staging of A_tj (2 x nkap)
  void* tab_xi[2];                // ny values of type T
  void* tab_cdf[2];               // ny x nkap values of type T
  int* tab_guide[2];              // FP32: ny x (kTabGuide + 1) guide-table entries
  unsigned long long* tab_xmax;   // the largest xi of each type
  // tangent mode (likelihood-ratio d/dH, d/dw; sp1, 2D)
  int tangent;
  long long tquantum;             // tangent particles carry |tau| <= tquantum 2^-32
  long long* dgrid[2];            // tangent histogram (H, w) of all instances, 2^-32 units
  uint32_t* tnz_cell;             // the tangent plan: cells with tangent weight,
  unsigned long long* tnz_start;  //   their first tangent slot,
  double* tnz_tau;                //   (tau_H, tau_w) of each of their particles,
  uint32_t* ttile_nz;             //   and the first plan entry of each 32-slot tile
  unsigned long long* tinst_slot; // first tangent slot of each instance (+ total)
  double* inst_grad;              // read-out (dT/dH, dT/dw) per instance (device)
  // time-dependent potential (wbrw_init_td): components on the device
  int ncomp;
  int lean;           // FP32 2D, static potential, no event log (tangents or not)
  void* comp_tab;
  // scratch carve-up
  Counters* cnt;
  unsigned long long* cpid;
  // queues, each with one private segment per producer warp: entries per
  // segment (*seg) and per-segment counts (*cnt)
  int nseg;
  void* fq[2];        // offspring waves (double buffered)
  unsigned* fcnt[2];
  long long qcap, qseg;
  void* eq[2];        // candidate intervals of the even and odd rounds
  unsigned* ecnt[2];
  long long ecap, eseg;
  void* dq[2];        // deferred segments, levels alternating
  unsigned* dcnt;     // kMaxLevels x kMaxSeg
  long long dcap, dseg;
  unsigned* rcnt;     // sp2 records per segment
  long long rseg;
  int max_chunk;      // steps per flight: about one candidate per particle
  Counters* cnt_save; // autotuner: the counters to put back
  int bps;            // tuning: resident blocks per SM of the queue kernels
  int max_bps;        // the most the context's kernels are built for (3 or 4)
  int passes;         // tuning: lockstep event passes before the drain
  uint32_t* nz_cell;
  unsigned long long* nz_start;
  uint32_t* tile_nz;  // first nonzero cell of each 32-slot tile of the plan
  long long tile_cap;
  unsigned long long* scan_bsum;
  unsigned int* scan_bnz;
  long long scan_blocks;
  int* tmp_grid;
  long long* tmp_wsum;
  double* obs_density;
  long long* obs_red;   // dim 4: counts summed over (x2, k2), nx x nk
  double* obs_marg;
  long long* obs_col;
  double* obs_scalar;
  uint32_t* rec_cell;
  uint32_t* rec_a;
  long long rec_cap;
  int* boot_keep[2];
  unsigned long long* boot_res[2];
  int* boot_ucnt;     // sp2: regenerated (unit-weight) particles per side and cell, 2 x nh
  int* boot_guide;    // sp2: 2 x (kGuide + 1) guide-table entries of the draws
  BootInst* boot_inst;             // sp2 batches: per-instance bootstrap records
  unsigned long long* boot_dpre;   //   and the exclusive prefix of their draws (2 ninst + 1)
  int* boot_bguide;                //   and their guide tables, 2 ninst x (kGuideB + 1)
  // state
  int state;  // 0 = particles in the arrays, 1 = histogram (grid + nz lists)
  long long step;
  long long epoch;
  int fresh;
  int failed;
  int capturing;      // a period is being captured into a CUDA graph
  int graph_on;       // wbrw_graph: replay periods from CUDA graphs
  int one_launch;     // wbrw_one_launch_periods: fused periods where the kernels allow
  int dev_period_ok;  // the device period state equals (step, epoch)
  int ngraphs;
  PeriodGraph graphs[kMaxGraphs];
  // placeholders of the captured event records: the first wave, then the
  // event kernel of each round
  cudaEvent_t gev[2 + 2 * kProfRounds];
  int gev_created;
  // the profiling events are recorded on a side stream that waits for the
  // context stream's work so far (in a captured period: a side branch,
  // joined before the capture ends), so that the kernels do not wait for
  // the records
  cudaStream_t prof_side;
  cudaEvent_t prof_fork, prof_join;
  int prof_side_used;     // the capture in progress forked the side stream
  int prof_side_created;
  long long launches;
  // CUDA-event timing of the first flight wave of each chunk (prof_ev) and
  // of each event-kernel launch (prof_evk)
  int prof_on;
  int prof_n, prof_nk;
  cudaEvent_t prof_ev[2 * kProfLaunches];
  cudaEvent_t prof_evk[2 * kProfLaunches];
  int prof_created;
  char err[512];
};

enum { ST_PARTICLES = 0, ST_HISTOGRAM = 1 };


// Per-precision drivers (wbrw_fp64.cu / wbrw_fp32.cu).
// Event pair around a profiled launch (no-ops while profiling is off):
// kind PROF_FIRST_WAVE, or PROF_EVENT with the launch's round r.
enum { PROF_FIRST_WAVE = 0, PROF_EVENT = 1 };
void prof_begin(Ctx*, int kind = PROF_FIRST_WAVE, int r = 0);
void prof_end(Ctx*, int kind = PROF_FIRST_WAVE, int r = 0);

struct Driver {
  cudaError_t (*init)(Ctx*, long long n);
  // Fly [l0, L) from the source, offspring in waves, finals to dst.
  cudaError_t (*chunk)(Ctx*, int l0, int L, int src, int dst);
  // Histogram the arrays (no flight): dst = DST_BIN1 into grid / DST_BIN2
  // records / DST_WSUM into tmp_wsum; count_ledger = tally out-of-grid.
  cudaError_t (*bin)(Ctx*, int dst, int* grid, int count_ledger);
  // Regenerate the histogram into the arrays (Alg. 3).
  cudaError_t (*materialize)(Ctx*);
  cudaError_t (*pids)(Ctx*, unsigned long long* out, unsigned* inst_out);
  // 4D model: build the kernel tables from A (host, 2 x nkap values) and
  // return the largest xi of each type (synchronises).
  cudaError_t (*tables)(Ctx*, const double* A_host, double* xmax_host);
  int fentry_bytes, sentry_bytes;  // queue entry sizes of this model and precision
  int max_bps;                     // resident blocks per SM its queue kernels are built for
  int inline_drain;                // its event kernel finishes deferred segments (no passes)
};

const Driver* driver_fp64();
const Driver* driver_fp32();
const Driver* driver_fp32_lean();
const Driver* driver_fp32_lean_batch();
const Driver* driver_fp32_grad_lean();
const Driver* driver_fp64_4d();
const Driver* driver_fp32_4d();
const Driver* driver_fp64_grad();
const Driver* driver_fp32_grad();

// Precision-independent launches (wbrw_common.cu).
cudaError_t launch_setup(Ctx*, int op, unsigned long long a,
                         unsigned long long b);
cudaError_t launch_scan_cells(Ctx*, const int* grid);
// The tangent plan from the tangent histogram (tangent mode).
cudaError_t launch_scan_tangent(Ctx*);
// (dT/dH, dT/dw) of every instance from the tangent histogram, into
// c->inst_grad.
cudaError_t launch_transmission_gradients(Ctx*);
// sp2: the bootstrap of the period's records and unit counts into the grid
// (a batch bootstraps every instance on its own).
cudaError_t launch_boot(Ctx*, int epoch_delta);
// wp: Alg. 3's rounding of the weighted histogram tmp_wsum into the grid.
cudaError_t launch_wp_round(Ctx*, int epoch_delta);
// Observables of instance `inst` from the counts / Q1.31 weight sums of all
// instances (one of the two is NULL).
cudaError_t launch_observables(Ctx*, int inst, const int* counts, const long long* wsum);
// Transmission of every instance into out (ninst doubles, device).
cudaError_t launch_transmissions(Ctx*, const int* counts, double* out);
cudaError_t launch_zero(Ctx*, void* p, size_t bytes);
// Materialised particles of instance `inst` (base region + offspring) added
// to *out (device).
cudaError_t launch_live_instance(Ctx*, int inst, unsigned long long* out);

// k_setup operations.  SETUP_PERIOD: set the device period state only.
// SETUP_CHUNK: snapshot n, set the chunk's first
// interval (a) and id base (b).  SETUP_CHUNK_DEV: snapshot n only (a captured
// period takes both from the device).  SETUP_ADVANCE: move the device period
// state on by a intervals and one resampling.  SETUP_AFTER_REGEN: the arrays
// hold the regeneration of id base a at interval b.
enum { SETUP_CHUNK = 0, SETUP_AFTER_REGEN = 1, SETUP_INIT = 2,
       SETUP_BOOT = 3, SETUP_CHUNK_DEV = 4, SETUP_ADVANCE = 5, SETUP_PERIOD = 6 };

}  // namespace wbrw
