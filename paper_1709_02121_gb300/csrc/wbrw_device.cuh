// wbrw_device.cuh -- device code of the signed-particle WBRW hot path for
// sm_103a (GB300), templated on the particle precision.
//
// One kernel, k_flight<P, SRC, DST>, carries the hot path of Alg. 1 (Xiong &
// Shao, arXiv:1709.02121) for a chunk of intervals [l0, L):
//   source  SRC_ARRAY  particles in the caller's SoA arrays
//           SRC_REGEN  Alg. 3 regeneration from the histogram, in registers
//           SRC_QUEUE  (FP64) offspring waiting at the start of a later interval
//   flight  free streaming x <- x + (hbar/m) k dt (Eq. 1) and the candidate
//           clock of constant rate gamma0 (Sec. 3.2): which intervals hold a
//           candidate event
//   sink    DST_ARRAY  back to the arrays (offspring appended)
//           DST_BIN1   signed histogram c_nu (Eq. signed_histogram)
//           DST_BIN2   (cell, |w| in Q1.31) records for the sp2 bootstrap
//           DST_WSUM   signed weights per cell in fixed point (wp, observables)
// Candidate intervals go to per-warp queue segments and round by round to
// k_event and its follow-up passes (one event per lane per pass): the kick of
// Remark 3, the acceptance (sp1) or weight (sp2/wp) cacc |sin|, the +/- pair
// of Alg. 1 item 3 and the offspring's own events in the same interval.  An
// FP32 offspring then flies on to the sink inside the event kernel, its
// candidate intervals queued for the next round; an FP64 offspring joins the
// next wave, a launch of k_flight with SRC_QUEUE (the FP64 clock draws per
// interval).  Every queue has one private segment per producer warp, so
// appending takes no global atomic, and no barrier is taken inside any main
// loop.
#pragma once

#include <cuda_runtime.h>
#include <cmath>
#include <type_traits>
#include <math_constants.h>
#include <stdint.h>
#include <string.h>

#include "wbrw_internal.h"

namespace wbrw {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11), written from its definition.
// ---------------------------------------------------------------------------
// The key schedule is precomputed on the host (the keys of round r are
// key + r * (0x9E3779B9, 0xBB67AE85)) and read from the kernel's parameter
// space.
struct KeySched {
  uint32_t k0[10], k1[10];
};

__device__ __forceinline__ uint4 philox_ks(const KeySched& ks, uint32_t c0, uint32_t c1,
                                           uint32_t c2, uint32_t c3) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ ks.k0[r];
    const uint32_t n2 = hi0 ^ c3 ^ ks.k1[r];
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  return __dmul_rn(__dadd_rn(__dmul_rn((double)(a >> 5), 67108864.0),
                             (double)(b >> 6)),
                   1.0 / 9007199254740992.0);
}
__device__ __forceinline__ float u24(uint32_t a) {
  return (float)(a >> 8) * (1.0f / 16777216.0f);
}

// Counter word 2 of the reserved (non-step) streams and the id-draw flag.
constexpr uint32_t kStepInit = 0xFFFFFFFFu;
constexpr uint32_t kStepRegen = 0xFFFFFFFEu;
constexpr uint32_t kStepBoot = 0xFFFFFFFDu;
constexpr uint32_t kStepRound = 0xFFFFFFFCu;
constexpr uint32_t kDrawPids = 0x80000000u;
constexpr uint32_t kDrawGap = 0xC0000000u;    // FP32 gap to the next candidate interval
constexpr uint32_t kDrawComp = 0x40000000u;   // component choice (time-dependent V)

// ---------------------------------------------------------------------------
// Precision traits.  FP64 arithmetic goes through the _rn intrinsics so that
// no multiply-add is contracted: every expression rounds exactly as written,
// which is the operation order the FP64 parity contract fixes.
// ---------------------------------------------------------------------------
struct F64 {
  using T = double;
  static constexpr bool is64 = true;
  __device__ static T add(T a, T b) { return __dadd_rn(a, b); }
  __device__ static T sub(T a, T b) { return __dsub_rn(a, b); }
  __device__ static T mul(T a, T b) { return __dmul_rn(a, b); }
  __device__ static T div(T a, T b) { return __ddiv_rn(a, b); }
  __device__ static T stream(T x, T k, T dtv) { return add(x, mul(k, dtv)); }
  __device__ static T flr(T a) { return floor(a); }
  __device__ static T next_dn(T a) { return nextafter(a, -CUDART_INF); }
  __device__ static T next_up(T a) { return nextafter(a, CUDART_INF); }
  __device__ static T sn(T a) { return sin(a); }
  __device__ static T cs(T a) { return cos(a); }
};

struct F32 {
  using T = float;
  static constexpr bool is64 = false;
  __device__ static T add(T a, T b) { return __fadd_rn(a, b); }
  __device__ static T sub(T a, T b) { return __fsub_rn(a, b); }
  __device__ static T mul(T a, T b) { return __fmul_rn(a, b); }
  __device__ static T div(T a, T b) { return __fdiv_rn(a, b); }
  __device__ static T stream(T x, T k, T dtv) { return __fmaf_rn(k, dtv, x); }
  __device__ static T flr(T a) { return floorf(a); }
  __device__ static T next_dn(T a) { return nextafterf(a, -CUDART_INF_F); }
  __device__ static T next_up(T a) { return nextafterf(a, CUDART_INF_F); }
  // sin and cos: the argument reduced to [-pi, pi] by Cody and Waite's
  // method (2 pi split into a head with 8 significant bits, so that n times
  // it is exact for |n| < 2^16, and a tail), then the hardware
  // approximation, whose absolute error on [-pi, pi] is below 2^-21.4; the
  // rounding of a phase argument of a few units already exceeds that
  __device__ static T reduce(T a) {
    const float n = rintf(a * 0.15915494f);
    return __fmaf_rn(-n, 0.0019353071795862320f, __fmaf_rn(-n, 6.28125f, a));
  }
  __device__ static T sn(T a) { return __sinf(reduce(a)); }
  __device__ static T cs(T a) { return __cosf(reduce(a)); }
  // -ln x for x in (0, 1]: the hardware logarithm (absolute error below
  // 2^-21.4 on [0.5, 2], at most 3 ulp elsewhere), clamped at 0 so that an
  // exponential variate never turns negative near x = 1.  Exponential and
  // geometric variates drawn from it differ from exact ones by less than
  // 4e-7 in -ln x, far below what the law tests resolve
  __device__ static T neg_ln(T x) { return fmaxf(-__logf(x), 0.0f); }
  // sqrt v for v >= 0 from the hardware reciprocal square root (a few ulp)
  __device__ static T sqrt_fast(T v) { return v > 0.0f ? v * rsqrtf(v) : 0.0f; }
};

// Phase-space model: precision F and D position coordinates (D = 1: the 2D
// phase space (x, k) of one particle; D = 2: the 4D phase space
// (x1, x2, k1, k2) of two electrons, Example 1).
//
// TGm: the tangent mode of the 2D model: every particle also carries its
// likelihood-ratio tangent weight (d/dH, d/dw), see do_event.
//
// LEANm: a run with the static potential and no event log: 1 for one
// instance, 2 for a batch.  The kernels then leave out the time-dependent
// components and the log writes, and for one instance the batch decode, and
// their registers (the results are those of the general kernels, which serve
// every other run).
template <class F, int Dm, bool TGm = false, int LEANm = 0>
struct PD : F {
  static constexpr int D = Dm;
  static constexpr bool TG = TGm;
  static constexpr bool LEAN = LEANm != 0;
  static constexpr bool SINGLE = LEANm == 1;  // one instance, known at compile time
};
using P64 = PD<F64, 1>;
using P32 = PD<F32, 1>;
using Q64 = PD<F64, 2>;
using Q32 = PD<F32, 2>;
using P64G = PD<F64, 1, true>;
using P32G = PD<F32, 1, true>;
using P32L = PD<F32, 1, false, 1>;
using P32LB = PD<F32, 1, false, 2>;
using P32GL = PD<F32, 1, true, 2>;  // tangent mode, static potential, no event log

// Resident 256-thread blocks per SM a queue kernel is built for (its launch
// bound).  The lean FP32 kernels and the FP32 4D kernels fit 64 registers,
// i.e. four blocks, without spilling or with little; the sp2 sink, the FP64,
// tangent and general FP32 kernels keep 80 registers and three blocks, which
// measured faster for them than four with spills.
template <class P, int DST>
__host__ __device__ constexpr int max_blocks() {
  return (!P::is64 && !P::TG && (P::LEAN || P::D == 2) && DST != DST_BIN2) ? 4 : 3;
}
template <class P>
__host__ __device__ constexpr int max_blocks_model() {
  return (!P::is64 && !P::TG && (P::LEAN || P::D == 2)) ? 4 : 3;
}
// The lean kernels and the FP32 4D ones finish their deferred segments
// inside the event kernel (k_event below) instead of in k_cont and k_drain
// launches ...
template <class P>
__host__ __device__ constexpr bool inline_drain() {
  return !P::is64 && (P::LEAN || (P::D == 2 && !P::TG));
}
// ... and run a regenerating period as one launch (k_period).
template <class P>
__host__ __device__ constexpr bool fused_period() {
  return inline_drain<P>();
}
static_assert(max_blocks_model<P32L>() <= kMaxBlocksPerSm, "tuning range");

// The tangent weight tau = s S (sign times lineage score) of a particle, in
// the run's precision (FP64 for the parity path; FP32 runs keep it in FP32,
// since FP64 arithmetic is slow on this GPU); an empty base outside the
// tangent mode.
template <bool TG, class U = double>
struct TanField {};
template <class U>
struct TanField<true, U> {
  U th, tw;
};
template <class P>
using TanOf = TanField<P::TG, typename P::T>;

// A position or a wavevector of the model.
template <class P>
struct PV {
  typename P::T c[P::D];
};

template <class P>
struct FEntry : TanOf<P> {  // a particle at the start of interval l (offspring
                                   // waves), or a candidate interval l with x at its start
  unsigned long long pid;
  PV<P> x, k;
  typename P::T w;
  int l;
};

static_assert(sizeof(FEntry<P64>) == 40 && sizeof(FEntry<P32>) == 24, "FEntry layout");
static_assert(sizeof(FEntry<P32L>) == sizeof(FEntry<P32>), "FEntry layout");
static_assert(sizeof(FEntry<P32LB>) == sizeof(FEntry<P32>), "FEntry layout");
static_assert(sizeof(FEntry<Q32>) == 32, "FEntry layout");
static_assert(sizeof(FEntry<P32G>) == 32 && sizeof(FEntry<P64G>) == 56, "FEntry layout");

template <class P>
struct SEntry;


// Physics of one instance of a batch (a single run is a batch of one).  In
// the 4D model gamma0 is the total rate Gamma of the three components.
template <class T>
struct Inst {
  T gamma0, cacc, sig_k, xc;  // rate, acceptance factor C/(2 gamma0), kick scale, centre
  double p_hi;                // FP64: u0 < p_hi may start an event in an interval
  float p_any_f;              // FP32: P(candidate) per interval
  float ilq;                  // FP32: 1 / ln(1 - p_any), the geometric gap's scale
  float ig0;                  // FP32: 1 / gamma0
  int well;                   // H < 0: V_W has the sign of -sin (Eq. 2)
  T gH, gw0, gw1;             // tangent mode: 1/H, 1/w, 4w (the score of a birth)
};

// Initial sampling of one instance: slots [start, start + n) of the arrays
// (x0b, k0b: the second electron of the 4D model).
struct InitInst {
  double x0, sx, k0, sk;
  unsigned long long start;
  double x0b, k0b;
};

// Kernel tables of the 4D model (type 0: one-body, 1: interaction).  Row i
// of type t belongs to y_i = -Y_t + i dy_t; cell j to kappa_j =
// -K + (j + 1/2) dkappa.  cdf rows: FP64 the prefix sums S_ij of V_W^+,
// FP32 S_ij / S_i,last.
template <class T>
struct Tab4 {
  const T* xi[2];     // ny per type
  const T* cdf[2];    // ny x nkap per type
  const int* guide[2];  // FP32: ny x (kTabGuide + 1) per type (see k_tab4_guide)
  double Y[2], inv_dy[2];
  double gam[2];      // component rates gamma_t (one-body twice, interaction once)
  double xc;          // nucleus
  T kap0, dkap;       // -K, dkappa
  int ny, nkap;
};

// Queue entries carry the interval and the instance in one word.
constexpr int kLBits = 24;
__device__ __forceinline__ int ent_l(int v) { return v & ((1 << kLBits) - 1); }
__device__ __forceinline__ int ent_inst(int v) { return (int)((unsigned)v >> kLBits); }
__device__ __forceinline__ int ent_pack(int l, int inst) { return l | (inst << kLBits); }

// Kernel parameters (by value, parameter space).
//
// Queues.  Every queue is split into one private segment per producer warp
// (nseg segments of *seg entries; warp g of any producing kernel owns
// segment g).  A producing warp keeps its running count in shared memory and
// writes it back once at the end of the kernel, so no global atomic is ever
// taken to append.  Kernels of one round that feed the same queue run one
// after the other and continue each other's counts.  Consumers walk the
// segments one warp at a time.
template <class P>
struct KP {
  using T = typename P::T;
  T dt, dtv, hm;
  T inv_dt;         // 1/dt
  T dt_lo;          // the largest value below dt
  Tab4<T> tab;      // 4D model only
  const Comp* comp; // time-dependent potential: ncomp components (0: static)
  int ncomp;
  T xmin, kmin, kmax, dx, dk, inv_dx, inv_dk;
  int nx, nk;
  float inv_nk;     // 1/nk, for cell -> (ix, ik)
  int nh_big;       // cells per instance >= 2^24: an integer division instead
  unsigned long long inst_mag;  // ceil(2^40 / nhi): the instance of a global cell
  int ninst;        // instances in the batch (1 for a single run)
  int nhi;          // cells per instance (nx nk); instance i owns [i nhi, (i+1) nhi)
  const Inst<T>* inst;                    // per-instance physics
  Inst<T> inst0;                          // instance 0's record, in the parameters
  const unsigned long long* inst_slot;    // first array slot of each base instance
  const unsigned long long* regen_start;  // first regenerated slot of each instance
  unsigned* cinst;                        // instance of offspring appended to the arrays
  KeySched ks;      // Philox key schedule of the run seed
  int strategy;     // 1 = sp1, 2 = sp2
  int l0, L;        // the intervals [l0, L) of the chunk (read at kernel entry)
  int len;          // L - l0
  unsigned long long regen_base;  // epoch << 40 of the histogram's particles
  T* x;             // coordinate d of slot i at x[d capacity + i]
  T* k;
  signed char* s;
  T* w;
  long long capacity;
  unsigned long long* cpid;
  int nseg;                  // segments per queue (producer warps)
  FEntry<P>* fq_in;          // offspring of the previous wave
  const unsigned* fcnt_in;
  FEntry<P>* fq_out;         // offspring for the next wave (FP64)
  unsigned* fcnt_out;
  unsigned qseg;
  FEntry<P>* eq;             // candidate intervals: the queue appended to
  FEntry<P>* eq_alt;         // the other candidate buffer (one-launch periods)
  unsigned* ecnt;
  const FEntry<P>* eq_in;    // the candidate intervals k_event takes
  const unsigned* ecnt_in;
  unsigned eseg;
  SEntry<P>* dq[2];          // deferred segments; level L lives in dq[L & 1]
  unsigned* dcnt;            // kMaxLevels x nseg counts
  unsigned dseg;
  uint32_t* rec_cell;        // sp2 records (cell | side << 31, |w| in Q1.31)
  uint32_t* rec_a;
  unsigned* rcnt;
  unsigned rseg;
  int* ucnt;                 // sp2: unit-weight particles per (side, cell of any instance),
                             // side-major (side stride nhi ninst)
  int* grid;
  long long* wsum;
  const uint32_t* nz_cell;
  const unsigned long long* nz_start;
  const uint32_t* tile_nz;   // first nonzero cell of each 32-slot tile
  long long tile_cap;
  // tangent mode: the tangent histogram D (2^-32 units) and tangent arrays
  // (slot i: tan[i] = tau_H, tan[capacity + i] = tau_w); the tangent
  // particles' plan: nonzero cells, first slots, tau per particle, tiles
  long long* dgrid[2];
  double* tan;
  const uint32_t* tnz_cell;
  const unsigned long long* tnz_start;
  const double* tnz_tau;     // (tau_H, tau_w) of each plan entry
  const uint32_t* ttile_nz;
  const unsigned long long* tinst_slot;
  Counters* cnt;
  wbrw_event* log;
  long long log_cap;
  int count_ledger;
};

// The chunk's first interval and the regeneration's id base are
// device-resident (Counters::per_*): the chunk set-up writes them, and a
// captured period advances them in place, so that one captured period replays
// correctly.  Each kernel takes them into its own copy of the parameters.
template <class P>
__device__ __forceinline__ KP<P> with_period(const KP<P>& q) {
  KP<P> p = q;
  p.l0 = q.cnt->per_l0;
  p.L = p.l0 + q.len;
  p.regen_base = q.cnt->per_regen_base;
  return p;
}

// The physics record of instance i: a single run reads it from the kernel
// parameters (constant bank), a batch from its table in global memory.
template <class P>
__device__ __forceinline__ Inst<typename P::T> inst_of(const KP<P>& p, int i) {
  if (!P::SINGLE && p.ninst > 1) return p.inst[i];
  return p.inst0;
}

constexpr int kWarps = kBlock / 32;
constexpr int kStack = 32;    // pending offspring frames per thread (drain)
constexpr unsigned kFull = 0xFFFFFFFFu;

// Per-thread tallies, reduced once per block at the end of a kernel.  The
// counts are 32-bit: a thread touches at most (its share of the capacity) x
// (the intervals of one flight, <= kMaxChunk) particle-steps in a launch,
// below 2^32 for every capacity the library accepts; the Q1.31 weight sums
// need 64 bits.
struct Acc {
  unsigned psteps, events, kill_p, kill_m, out_p, out_m;
  unsigned n_plus, n_minus;
  unsigned long long w_plus, w_minus;
  unsigned cand;  // first events of candidate intervals (k_event)
  __device__ void zero() {
    psteps = events = kill_p = kill_m = out_p = out_m = 0;
    n_plus = n_minus = w_plus = w_minus = 0;
    cand = 0;
  }
};

// A warp's running counts in the queues it produces into; flip selects the
// candidate buffer it appends to (p.eq, or p.eq_alt in the rounds of a
// one-launch period).
struct WarpCounts {
  unsigned f, e, d, r, flip;
};

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_err(Counters* c, int bit) {
  atomicOr(&c->err, bit);
}

__device__ __forceinline__ unsigned global_warp() {
  return blockIdx.x * kWarps + (threadIdx.x >> 5);
}

// The histogram cell of a phase-space point (Sec. 4.3, uniform mesh):
// ix nk + ik, or ((ix1 nx + ix2) nk + ik1) nk + ik2 in the 4D model.
template <class P>
__device__ __forceinline__ bool cell_of(const KP<P>& p, const PV<P>& x, const PV<P>& k,
                                        int& cell) {
  using T = typename P::T;
  int ix[P::D], ik[P::D];
#pragma unroll
  for (int d = 0; d < P::D; ++d) {
    const T fx = P::flr(P::mul(P::sub(x.c[d], p.xmin), p.inv_dx));
    const T fk = P::flr(P::mul(P::sub(k.c[d], p.kmin), p.inv_dk));
    if (!(fx >= (T)0 && fx < (T)p.nx && fk >= (T)0 && fk < (T)p.nk)) return false;
    ix[d] = (int)fx;
    ik[d] = (int)fk;
  }
  if constexpr (P::D == 1) cell = ix[0] * p.nk + ik[0];
  else cell = ((ix[0] * p.nx + ix[1]) * p.nk + ik[0]) * p.nk + ik[1];
  return true;
}

// Position at time t of a segment that started at (xo, to).
template <class P>
__device__ __forceinline__ PV<P> pos_at(const KP<P>& p, const PV<P>& xo,
                                        typename P::T to, const PV<P>& k, typename P::T t) {
  PV<P> x;
  const typename P::T h = P::mul(P::sub(t, to), p.hm);
#pragma unroll
  for (int d = 0; d < P::D; ++d) x.c[d] = P::add(xo.c[d], P::mul(k.c[d], h));
  return x;
}

template <class P>
__device__ __forceinline__ bool k_inside(const KP<P>& p, const PV<P>& k) {
  bool in = true;
#pragma unroll
  for (int d = 0; d < P::D; ++d) in = in && k.c[d] >= p.kmin && k.c[d] < p.kmax;
  return in;
}

// Sum of one value over the block, added to a global counter by one thread.
__device__ __forceinline__ void block_reduce_add(unsigned long long* red, unsigned long long v,
                                                 unsigned long long* dst) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int i = 0; i < kWarps; ++i) t += red[i];
    if (t) atomicAdd(dst, t);
  }
}

template <class P>
__device__ __forceinline__ void load_counts(const KP<P>& p, WarpCounts& wc, int level_out) {
  const unsigned g = global_warp();
  if ((threadIdx.x & 31) == 0) {
    const bool own = g < (unsigned)p.nseg;
    wc.f = own && p.fcnt_out ? p.fcnt_out[g] : 0u;
    wc.e = own && p.ecnt ? p.ecnt[g] : 0u;
    wc.d = own && level_out > 0 ? p.dcnt[(long long)level_out * p.nseg + g] : 0u;
    wc.r = own && p.rcnt ? p.rcnt[g] : 0u;
    wc.flip = 0u;
  }
  __syncwarp();
}

template <class P>
__device__ __forceinline__ void store_counts(const KP<P>& p, const WarpCounts& wc, int level_out,
                                             bool f, bool e, bool r) {
  __syncwarp();
  const unsigned g = global_warp();
  if ((threadIdx.x & 31) == 0 && g < (unsigned)p.nseg) {
    if (f && p.fcnt_out) p.fcnt_out[g] = wc.f;
    if (e && p.ecnt) p.ecnt[g] = wc.e;
    if (level_out > 0) p.dcnt[(long long)level_out * p.nseg + g] = wc.d;
    if (r && p.rcnt) p.rcnt[g] = wc.r;
  }
}

// ---------------------------------------------------------------------------
// Per-precision draws.  A "segment" is a particle's part of interval l from
// time `to` on (0 for a particle present at t_l, its birth time for an
// offspring).  Draw<P>::first gives the time of the segment's first event
// (>= dt when there is none); Draw<P>::event gives event j's kick, sign
// factor, acceptance uniform and next gap.
// ---------------------------------------------------------------------------
template <class P, bool = P::is64>
struct Draw;

// The kick of the 4D model from its tables, given the event's uniforms:
// component m (0: y = x1 - xc on k1; 1: y = x2 - xc on k2; 2: y = x1 - x2
// on (k1, -k2)) is the first with uc Gamma < gamma_0 + ... + gamma_m; the row
// position s = (y + Y)/dy, clamped to the mesh, splits into node i and weight
// th; with g0 = (1 - th) xi_i and g1 = th xi_{i+1} the pair comes from row i
// if ua gamma_m < g0, from row i+1 if ua gamma_m < g0 + g1, and is not made
// otherwise, which thins the rate gamma_m down to the interpolant xi_h(y)
// (Sec. 3.2, Eq. def.xi_m) and makes the kick law the interpolant of the two
// rows' laws.  The kick is kappa_j + (uj - 1/2) dkappa for the first cell j
// of the row's inverse CDF above uk.  prob = xi_h(y)/gamma_m.
template <class P>
__device__ __forceinline__ bool table_kick(const KP<P>& p, typename P::T Gam, const PV<P>& xe,
                                           typename P::T ua, typename P::T uk,
                                           typename P::T uc, typename P::T uj, int& comp,
                                           typename P::T& kap, typename P::T& prob) {
  using T = typename P::T;
  const Tab4<T>& tb = p.tab;
  const T g_ne = (T)tb.gam[0], g_ee = (T)tb.gam[1];
  const T v = P::mul(uc, Gam);
  const int m = v < g_ne ? 0 : (v < P::mul((T)2, g_ne) ? 1 : 2);
  comp = m;
  const int t = m == 2 ? 1 : 0;
  const T xc = (T)tb.xc;
  const T y = m == 0 ? P::sub(xe.c[0], xc)
                     : (m == 1 ? P::sub(xe.c[P::D - 1], xc) : P::sub(xe.c[0], xe.c[P::D - 1]));
  const T g = m == 2 ? g_ee : g_ne;
  // (selects, not indexing by t: the parameters stay out of local memory)
  const T sp = P::mul(P::add(y, (T)(t ? tb.Y[1] : tb.Y[0])), (T)(t ? tb.inv_dy[1] : tb.inv_dy[0]));
  int i;
  T th;
  if (!(sp > (T)0)) {
    i = 0;
    th = (T)0;
  } else if (sp >= (T)(tb.ny - 1)) {
    i = tb.ny - 2;
    th = (T)1;
  } else {
    i = (int)P::flr(sp);
    th = P::sub(sp, (T)i);
  }
  const T* xi = t ? tb.xi[1] : tb.xi[0];
  const T g0 = P::mul(P::sub((T)1, th), xi[i]);
  const T g1 = P::mul(th, xi[i + 1]);
  const T g01 = P::add(g0, g1);
  prob = g > (T)0 ? P::div(g01, g) : (T)0;
  const T va = P::mul(ua, g);
  int r;
  if (va < g0) r = i;
  else if (va < g01) r = i + 1;
  else return false;
  const T* row = (t ? tb.cdf[1] : tb.cdf[0]) + (long long)r * tb.nkap;
  const T target = P::is64 ? P::mul(uk, row[tb.nkap - 1]) : uk;
  int lo = 0, hi = tb.nkap - 1;  // the first cell whose cumulative sum exceeds target
  if constexpr (!P::is64) {
    // FP32 rows are normalised: uk (on the 2^-24 grid) lies in bucket
    // b = floor(uk 2^kTabGuideBits) exactly, and the answer in
    // [G_b, G_(b+1)] of the row's guide table: the same cell as the full search
    const int b = (int)(uk * (float)kTabGuide);
    const int* gd = (t ? tb.guide[1] : tb.guide[0]) + (long long)r * (kTabGuide + 1);
    lo = gd[b];
    hi = gd[b + 1];
  }
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (row[mid] > target) hi = mid;
    else lo = mid + 1;
  }
  const T kj = P::add(tb.kap0, P::mul(P::add((T)lo, (T)0.5), tb.dkap));
  kap = P::add(kj, P::mul(P::sub(uj, (T)0.5), tb.dkap));
  return true;
}

// FP64: the parity contract shared with the oracle.  u0 of (pid, l, 0)
// gives the first life-length from `to`; event j uses (pid, l, 1+2j) and
// (pid, l, 2+2j).  Offspring draw their first life-length the same way.
// In the 4D model event j takes from those two calls ua = U53(a0,a1),
// uk = U53(a2,a3), the gap from U53(b0,b1), uc = b2 2^-32, uj = b3 2^-32.
template <class P>
struct Draw<P, true> {
  struct State {};
  __device__ static double first(const KP<P>& p, const Inst<double>& ip,
                                 unsigned long long pid, int l, double to, bool /*root*/,
                                 State&) {
    const uint4 r = philox_ks(p.ks, (uint32_t)pid, (uint32_t)(pid >> 32), (uint32_t)l, 0u);
    const double u0 = u53(r.x, r.y);
    return P::add(to, P::div(-log1p(-u0), ip.gamma0));
  }
  __device__ static bool event4(const KP<P>& p, const Inst<double>& ip, unsigned long long pid,
                                int l, unsigned j, const PV<P>& xe, const State&, int& comp,
                                double& kap, double& prob, double& gap) {
    const uint32_t lo = (uint32_t)pid, hi = (uint32_t)(pid >> 32);
    const uint4 a = philox_ks(p.ks, lo, hi, (uint32_t)l, 1u + 2u * j);
    const uint4 b = philox_ks(p.ks, lo, hi, (uint32_t)l, 2u + 2u * j);
    const double ua = u53(a.x, a.y), uk = u53(a.z, a.w), ug = u53(b.x, b.y);
    const double uc = (double)b.z * (1.0 / 4294967296.0);
    const double uj = (double)b.w * (1.0 / 4294967296.0);
    gap = __ddiv_rn(-log1p(-ug), ip.gamma0);
    return table_kick<P>(p, ip.gamma0, xe, ua, uk, uc, uj, comp, kap, prob);
  }
  // event j of the 2D model: the standard normal z of the kick, the
  // acceptance uniform u3 and the gap to the next event
  __device__ static void event(const KP<P>& p, const Inst<double>& ip, unsigned long long pid,
                               int l, unsigned j, bool /*root*/, const State&, double& z,
                               double& u3, double& gap) {
    const uint32_t lo = (uint32_t)pid, hi = (uint32_t)(pid >> 32);
    const uint4 a = philox_ks(p.ks, lo, hi, (uint32_t)l, 1u + 2u * j);
    const uint4 b = philox_ks(p.ks, lo, hi, (uint32_t)l, 2u + 2u * j);
    const double u1 = u53(a.x, a.y), u2 = u53(a.z, a.w);
    u3 = u53(b.x, b.y);
    const double u4 = u53(b.z, b.w);
    z = __dmul_rn(__dsqrt_rn(__dmul_rn(-2.0, log1p(-u1))),
                  cos(__dmul_rn(6.283185307179586476925286766559, u2)));
    gap = __ddiv_rn(-log1p(-u4), ip.gamma0);
  }
};

// FP32: the production contract, checked in law.
//  - Root segments (the interval is a known candidate): one call (pid, l, 0)
//    serves both the first life-length, drawn from the exponential truncated
//    to the interval, tau = -log1p(-p_any U24(w0))/gamma0, and event 0
//    (u1..u3 = U24(w1..w3), u4 from the low bytes of w0..w2).
//  - Offspring segments (from their birth time tb): the first event comes at
//    tb + E/gamma0, E = -ln U exponential (memorylessness), U = (2m + 1)
//    2^-24 from bits 9..31 of the offspring's own random id; no event in the
//    interval when that time is >= dt.
//  - Event j of a segment, except event 0 of a root, uses the call
//    (pid, l, 1+j): u1..u4 = U24 of w0..w3.
//  - In the 4D model every event j, the first included, uses the call
//    (pid, l, 1+j): ua = U24(w0), uk = U24(w1), the gap from U24(w2),
//    uc = (w3 >> 16) 2^-16, uj = (w3 & 0xFFFF) 2^-16.
template <class P>
struct Draw<P, false> {
  struct State {
    uint4 r;
  };
  __device__ static bool event4(const KP<P>& p, const Inst<float>& ip, unsigned long long pid,
                                int l, unsigned j, const PV<P>& xe, const State&, int& comp,
                                float& kap, float& prob, float& gap) {
    const uint4 a = philox_ks(p.ks, (uint32_t)pid, (uint32_t)(pid >> 32), (uint32_t)l, 1u + j);
    const float uc = (float)(a.w >> 16) * (1.0f / 65536.0f);
    const float uj = (float)(a.w & 0xFFFFu) * (1.0f / 65536.0f);
    gap = F32::neg_ln(1.0f - u24(a.z)) * ip.ig0;  // 1 - u exact on the 2^-24 grid
    return table_kick<P>(p, ip.gamma0, xe, u24(a.x), u24(a.y), uc, uj, comp, kap, prob);
  }
  __device__ static float first(const KP<P>& p, const Inst<float>& ip, unsigned long long pid,
                                int l, float to, bool root, State& st) {
    if (!root) {
      const float u = (float)(2u * ((uint32_t)pid >> 9) + 1u) * (1.0f / 16777216.0f);
      return to + F32::neg_ln(u) * ip.ig0;
    }
    st.r = philox_ks(p.ks, (uint32_t)pid, (uint32_t)(pid >> 32), (uint32_t)l, 0u);
    // below dt in exact arithmetic; kept below it after rounding
    return fminf(to + F32::neg_ln(__fmaf_rn(-ip.p_any_f, u24(st.r.x), 1.0f)) * ip.ig0, p.dt_lo);
  }
  __device__ static void event(const KP<P>& p, const Inst<float>& ip, unsigned long long pid,
                               int l, unsigned j, bool root, const State& st, float& z,
                               float& u3, float& gap) {
    float u1, u2, u4;
    if (j == 0 && root) {
      const uint4 r = st.r;
      u1 = u24(r.y);
      u2 = u24(r.z);
      u3 = u24(r.w);
      u4 = (float)(((r.x & 0xFFu) << 16) | ((r.y & 0xFFu) << 8) | (r.z & 0xFFu)) *
           (1.0f / 16777216.0f);
    } else {
      const uint4 a = philox_ks(p.ks, (uint32_t)pid, (uint32_t)(pid >> 32), (uint32_t)l, 1u + j);
      u1 = u24(a.x);
      u2 = u24(a.y);
      u3 = u24(a.z);
      u4 = u24(a.w);
    }
    // Box-Muller with the angle 2 pi (u2 - 1/2) in [-pi, pi) (law unchanged)
    // (u1, u4 lie on the 2^-24 grid of [0, 1): 1 - u is exact, and neg_ln
    // keeps an absolute error below 2^-21.4 there)
    z = F32::sqrt_fast(2.0f * F32::neg_ln(1.0f - u1)) * __cosf(6.2831855f * (u2 - 0.5f));
    gap = F32::neg_ln(1.0f - u4) * ip.ig0;
  }
};

// ---------------------------------------------------------------------------
// Sinks
// ---------------------------------------------------------------------------
template <class P>
__device__ __forceinline__ uint32_t q131(typename P::T w) {
  // |w| in Q1.31 (|w| <= 1): floor(|w| 2^31); scaling by 2^31 is exact in
  // either precision and the conversion truncates
  if constexpr (P::is64) return (uint32_t)floor(fabs(w) * 2147483648.0);
  else return (uint32_t)(fabsf(w) * 2147483648.0f);
}

// A weight in the fixed-point units 2^-31 of the wp histogram, rounded to
// nearest.  The scaling by 2^31 is exact in either precision, so the FP32
// form (no FP64 arithmetic) gives the same integer as the FP64 one.
template <class P>
__device__ __forceinline__ long long wsum_units(typename P::T w) {
  if constexpr (P::is64) return llrint(w * 2147483648.0);
  else return __float2ll_rn(w * 2147483648.0f);
}

// A particle outside the grid at binning: dropped and tallied by sign.  A
// non-finite coordinate also lands here (every comparison of the cell test
// fails for NaN or infinity), so this rare branch is where the numeric
// error is latched; the in-grid path pays nothing for the check.
template <class P>
__device__ __forceinline__ void tally_out(const KP<P>& p, Acc& acc, typename P::T w,
                                          const PV<P>& x, const PV<P>& k) {
  bool finite = true;
#pragma unroll
  for (int d = 0; d < P::D; ++d) finite = finite && isfinite(x.c[d]) && isfinite(k.c[d]);
  if (!finite) set_err(p.cnt, ERR_NUMERIC);
  if (p.count_ledger) {
    if (w > (typename P::T)0) ++acc.out_p;
    else if (w < (typename P::T)0) ++acc.out_m;
  }
}

// Tangent mode: tau into the tangent histogram, rounded to a multiple of
// 2^-32 so that the sums are exact and independent of order.
template <class P>
__device__ __forceinline__ void add_tangent(const KP<P>& p, long long gcell,
                                            const TanOf<P>& tau) {
  if constexpr (P::TG) {
    if (!p.dgrid[0]) return;
    // (scaling by 2^32 is exact in either precision)
    long long a, b;
    if constexpr (P::is64) {
      a = __double2ll_rn(tau.th * 4294967296.0);
      b = __double2ll_rn(tau.tw * 4294967296.0);
    } else {
      a = __float2ll_rn(tau.th * 4294967296.0f);
      b = __float2ll_rn(tau.tw * 4294967296.0f);
    }
    if (a) atomicAdd((unsigned long long*)(p.dgrid[0] + gcell), (unsigned long long)a);
    if (b) atomicAdd((unsigned long long*)(p.dgrid[1] + gcell), (unsigned long long)b);
  }
}

template <class P>
__device__ __forceinline__ void put_record(const KP<P>& p, Acc& acc, long long idx, int cell,
                                           typename P::T w) {
  const uint32_t a = q131<P>(w);
  p.rec_cell[idx] = (uint32_t)cell | (w < (typename P::T)0 ? 0x80000000u : 0u);
  p.rec_a[idx] = a;
  if (w > (typename P::T)0) { ++acc.n_plus; acc.w_plus += a; } else { ++acc.n_minus; acc.w_minus += a; }
}

// An end-of-chunk state produced inside the divergent event code.
template <class P, int DST>
__device__ void emit_child_final(const KP<P>& p, WarpCounts& wc, Acc& acc, int inst,
                                 unsigned long long pid, const PV<P>& x, const PV<P>& k,
                                 typename P::T w, const TanOf<P>& tau) {
  using T = typename P::T;
  int cell;
  const int cbase = inst * p.nhi;
  if constexpr (DST == DST_BIN1) {
    if (cell_of<P>(p, x, k, cell)) {
      if (!P::TG || w != (T)0) atomicAdd(p.grid + cbase + cell, w > (T)0 ? 1 : -1);
      add_tangent<P>(p, (long long)cbase + cell, tau);
    } else {
      tally_out<P>(p, acc, w, x, k);
    }
  } else if constexpr (DST == DST_WSUM) {
    if (cell_of<P>(p, x, k, cell))
      atomicAdd((unsigned long long*)(p.wsum + cbase + cell),
                (unsigned long long)wsum_units<P>(w));
    else tally_out<P>(p, acc, w, x, k);
  } else if constexpr (DST == DST_BIN2) {
    if (!cell_of<P>(p, x, k, cell)) { tally_out<P>(p, acc, w, x, k); return; }
    if (w == (T)0) return;
    const unsigned g = global_warp();
    const unsigned r = atomicAdd(&wc.r, 1u);
    if (g >= (unsigned)p.nseg || r >= p.rseg) {
      set_err(p.cnt, ERR_CAP_RECORDS);
      return;
    }
    put_record<P>(p, acc, (size_t)g * p.rseg + r, cbase + cell, w);
  } else {  // DST_ARRAY
    const unsigned long long slot = atomicAdd(&p.cnt->n, 1ull);
    if (slot >= (unsigned long long)p.capacity) { set_err(p.cnt, ERR_CAP_PARTICLES); return; }
#pragma unroll
    for (int d = 0; d < P::D; ++d) {
      p.x[d * p.capacity + slot] = x.c[d];
      p.k[d * p.capacity + slot] = k.c[d];
    }
    p.s[slot] = w > (T)0 ? 1 : (w < (T)0 ? -1 : 0);
    if (p.w) p.w[slot] = w;
    if constexpr (P::TG) {
      p.tan[slot] = tau.th;
      p.tan[p.capacity + slot] = tau.tw;
    }
    p.cpid[slot - p.cnt->n_base] = pid;
    if (!P::SINGLE && p.ninst > 1) p.cinst[slot - p.cnt->n_base] = (unsigned)inst;
  }
}

// ---------------------------------------------------------------------------
// Events (Alg. 1 item 3).  A segment is a particle's part of interval l from
// time `to` (0 for a particle present at t_l, its birth time for an
// offspring).  Processing is split into passes so that the lanes of a warp
// follow the same path: each pass performs ONE event of each of its
// segments; a segment with another event left in the interval, and an
// offspring born with an event of its own, are deferred to the next pass.
// Offspring with no event left are settled at once: appended to the next
// wave, or sent to the sink in the chunk's last interval.  After the last
// pass a drain kernel finishes whatever remains with a full recursion.
// ---------------------------------------------------------------------------
template <class P>
struct SEntry : TanOf<P> {  // a deferred segment, with the time and index of its next event
  using T = typename P::T;
  unsigned long long pid;
  PV<P> xo;
  T to;
  PV<P> k;
  T w, t;
  int l;
  unsigned j;   // bits 0..30: index of the next event; bit 31: the root segment
  typename Draw<P>::State st;
};

static_assert(sizeof(SEntry<P64>) == 64 && sizeof(SEntry<P32>) == 64, "SEntry layout");
static_assert(sizeof(SEntry<P32L>) == 64 && sizeof(SEntry<P32LB>) == 64, "SEntry layout");
static_assert(sizeof(SEntry<Q32>) == 64, "SEntry layout");
static_assert(sizeof(SEntry<P32G>) == 64, "SEntry layout");

constexpr unsigned kRootFlag = 0x80000000u;

// FP32 candidate clock.  Whether an interval holds a candidate is a
// Bernoulli(p_any) trial, independent across intervals (the constant-rate
// clock of Sec. 3.2), so the number of whole intervals before the next
// candidate is geometric: G = floor(ln U / ln(1 - p_any)), U = (2 m + 1)
// 2^-24 from 23 random bits m.  Returns min(G, nmax).
__device__ __forceinline__ int geo_gap(uint32_t m, float ilq, int nmax) {
  const float u = (float)(2u * m + 1u) * (1.0f / 16777216.0f);
  const float g = __fmul_rn(-F32::neg_ln(u), ilq);
  return g < (float)nmax ? (int)g : nmax;
}

// Position after n free-flight intervals of length dt (dtv = dt hbar/m).
// FP64 rounds once per interval, in the oracle's order; FP32 takes the
// n intervals in one fused step, x + k (n dtv).
template <class P>
__device__ __forceinline__ typename P::T stream_n(typename P::T x, typename P::T k,
                                                  typename P::T dtv, int n) {
  if constexpr (P::is64) {
    for (int i = 0; i < n; ++i) x = P::stream(x, k, dtv);
    return x;
  } else {
    return n > 0 ? __fmaf_rn(k, __fmul_rn((float)n, dtv), x) : x;
  }
}

// FP32 candidate clock, continued by a root segment (a particle in one of
// its candidate intervals l) whose next event time t falls at or beyond dt:
// under the constant rate that event lies in interval l + floor(t/dt), the
// particle's next candidate interval, queued for the next round when it is
// inside the chunk.  Its own first event there is drawn afresh when that
// entry is taken (the interval's truncated exponential; memorylessness).
template <class P>
__device__ __forceinline__ void chain_next(const KP<P>& p, WarpCounts& wc,
                                           const SEntry<P>& s) {
  if constexpr (!P::is64) {
    const int l = ent_l(s.l);
    const float q = fmaxf(floorf(s.t * p.inv_dt), 1.0f);  // s.t >= dt
    if (q < (float)(p.L - l)) {
      const int c = l + (int)q;
      const unsigned g = global_warp();
      const unsigned slot = atomicAdd(&wc.e, 1u);
      if (g < (unsigned)p.nseg && slot < p.eseg) {
        FEntry<P> e;
        static_cast<TanOf<P>&>(e) = static_cast<const TanOf<P>&>(s);
        e.pid = s.pid;
#pragma unroll
        for (int d = 0; d < P::D; ++d) e.x.c[d] = stream_n<P>(s.xo.c[d], s.k.c[d], p.dtv, c - l);
        e.k = s.k;
        e.w = s.w;
        e.l = ent_pack(c, ent_inst(s.l));
        (wc.flip ? p.eq_alt : p.eq)[(size_t)g * p.eseg + slot] = e;
      } else {
        set_err(p.cnt, ERR_CAP_EQUEUE);
      }
    }
  }
}

// An offspring's state at the end of interval l: the next wave's input, or
// the sink's in the chunk's last interval.  t_next (>= dt) is the time of
// its next event under the constant-rate clock.
template <class P, int DST>
__device__ __forceinline__ void settle(const KP<P>& p, WarpCounts& wc, Acc& acc, int inst,
                                       unsigned long long pid, const PV<P>& xo,
                                       typename P::T to, const PV<P>& k, typename P::T w,
                                       int l, const TanOf<P>& tau,
                                       typename P::T t_next) {
  const PV<P> xf = pos_at(p, xo, to, k, p.dt);
  if constexpr (!P::is64) {
    // FP32: the offspring's flight through [l + 1, L) right here.  Its
    // next event lies in interval l + floor(t_next/dt), its first candidate
    // interval (as for a root, chain_next), queued for the next round when
    // inside the chunk; then the sink at the end of the chunk
    const int n = p.L - l - 1;
    if (n > 0) {
      acc.psteps += (unsigned)n;
      const float q = fmaxf(floorf(t_next * p.inv_dt), 1.0f);
      const int c = q < (float)(n + 1) ? l + (int)q : p.L;
      if (c < p.L) {
        const unsigned g = global_warp();
        const unsigned q = atomicAdd(&wc.e, 1u);
        if (g < (unsigned)p.nseg && q < p.eseg) {
          FEntry<P> e;
          static_cast<TanOf<P>&>(e) = tau;
          e.pid = pid;
#pragma unroll
          for (int d = 0; d < P::D; ++d) e.x.c[d] = stream_n<P>(xf.c[d], k.c[d], p.dtv, c - l - 1);
          e.k = k;
          e.w = w;
          e.l = ent_pack(c, inst);
          (wc.flip ? p.eq_alt : p.eq)[(size_t)g * p.eseg + q] = e;
        } else {
          set_err(p.cnt, ERR_CAP_EQUEUE);
        }
      }
      PV<P> xl;
#pragma unroll
      for (int d = 0; d < P::D; ++d) xl.c[d] = stream_n<P>(xf.c[d], k.c[d], p.dtv, n);
      emit_child_final<P, DST>(p, wc, acc, inst, pid, xl, k, w, tau);
    } else {
      emit_child_final<P, DST>(p, wc, acc, inst, pid, xf, k, w, tau);
    }
    return;
  }
  if (l + 1 < p.L) {
    FEntry<P> e;
    static_cast<TanOf<P>&>(e) = tau;
    e.pid = pid;
    e.x = xf;
    e.k = k;
    e.w = w;
    e.l = ent_pack(l + 1, inst);
    const unsigned g = global_warp();
    const unsigned q = atomicAdd(&wc.f, 1u);
    if (g < (unsigned)p.nseg && q < p.qseg)
      p.fq_out[(size_t)g * p.qseg + q] = e;
    else
      set_err(p.cnt, ERR_CAP_QUEUE);
  } else {
    emit_child_final<P, DST>(p, wc, acc, inst, pid, xf, k, w, tau);
  }
}

// Append a segment to the deferred level `level` (the one the kernel feeds).
template <class P>
__device__ __forceinline__ void defer(const KP<P>& p, WarpCounts& wc, int level,
                                      const SEntry<P>& s) {
  const unsigned g = global_warp();
  const unsigned q = atomicAdd(&wc.d, 1u);
  if (g < (unsigned)p.nseg && q < p.dseg)
    ((level & 1) ? p.dq[1] : p.dq[0])[(size_t)g * p.dseg + q] = s;
  else
    set_err(p.cnt, ERR_CAP_EQUEUE);
}

// A time-dependent potential (Remark 1): component m with probability
// gam_m/Gamma (uniform of the draw (pid, l, COMP | j)), its height
// H_m(t_l + t) at the event's absolute time, the kick sig_k,m z and the
// acceptance |H_m|/(hbar gam_m) |sin(2 (xe - xc_m) kappa)|, oriented by the
// sign of H_m sin.
template <class P>
__device__ __forceinline__ void comp_kick(const KP<P>& p, const Inst<typename P::T>& ip,
                                          unsigned long long pid, int l, unsigned j,
                                          typename P::T xe, typename P::T t, typename P::T z,
                                          typename P::T& kap, typename P::T& sg,
                                          typename P::T& fac, bool& flip) {
  using T = typename P::T;
  const uint4 c = philox_ks(p.ks, (uint32_t)pid, (uint32_t)(pid >> 32), (uint32_t)l, kDrawComp | j);
  T uc;
  if constexpr (P::is64) uc = u53(c.x, c.y);
  else uc = u24(c.x);
  const T v = P::mul(uc, ip.gamma0);
  int m = 0;
  T acc = (T)p.comp[0].gam;
  while (m + 1 < p.ncomp && !(v < acc)) {
    ++m;
    acc = P::add(acc, (T)p.comp[m].gam);
  }
  const Comp& q = p.comp[m];
  const T ta = P::add(P::mul((T)l, p.dt), t);
  const T Hm = P::add((T)q.a, P::mul((T)q.b, P::cs(P::add(P::mul((T)q.om, ta), (T)q.ph))));
  kap = P::mul((T)q.sig_k, z);
  sg = P::sn(P::mul(P::mul((T)2, P::sub(xe, (T)q.xc)), kap));
  fac = q.gam > 0.0 ? P::mul(P::div((T)fabs(Hm), (T)q.hg), (T)fabs(sg)) : (T)0;
  flip = Hm < (T)0 ? sg > (T)0 : sg < (T)0;
}

// An accepted event: what its +/- pair needs (the parent's id, tangent
// weight and weight, the event's position and time, the two wavevectors).
// 16-byte aligned for vector shared-memory loads, except with tangents: the
// per-warp buffers of the event kernels must stay within the 48 KB of static
// shared memory a block may declare (64 records of 56 bytes rather than 64).
template <class P>
struct alignas(P::TG ? 8 : 16) Birth : TanOf<P> {
  using T = typename P::T;
  unsigned long long pid;
  PV<P> xe, kp, km;
  T t, w, fac, kap;
  int l;       // interval | instance << kLBits
  unsigned j;  // the event's index in its segment
  int comp;    // 4D: the component
};

// Event j of a segment at time t, up to the decision.  2D model: the kick
// of Remark 3, the acceptance (sp1) or weight (sp2/wp) cacc |sin|, the +/-
// wavevectors.  4D model: the component, thinning and tabulated kick of
// table_kick; the pair is k +/- kappa e_m with e_0 = (1, 0), e_1 = (0, 1),
// e_2 = (1, -1).  Returns whether a pair is made (its data in b) and sets
// the gap to the segment's next event.
template <class P>
__device__ __forceinline__ bool event_decide(const KP<P>& p, const Inst<typename P::T>& ip,
                                             int inst, unsigned long long pid,
                                             const PV<P>& xo, typename P::T to,
                                             const PV<P>& k, typename P::T w,
                                             const typename Draw<P>::State& st, int l,
                                             unsigned j, bool root, typename P::T t,
                                             const TanOf<P>& tau, Birth<P>& b,
                                             typename P::T& gap) {
  using T = typename P::T;
  const PV<P> xe = pos_at(p, xo, to, k, t);
  T kap, fac;
  bool emit;
  int comp = 0;
  PV<P> kp = k, km = k;
  if constexpr (P::D == 1) {
    T z, sg, u3;
    bool flip;
    Draw<P>::event(p, ip, pid, l, j, root, st, z, u3, gap);
    if (P::LEAN || p.ncomp == 0) {  // the static barrier: kick, |sin| ratio, orientation
      kap = P::mul(ip.sig_k, z);
      sg = P::sn(P::mul(P::mul((T)2, P::sub(xe.c[0], ip.xc)), kap));
      fac = P::mul(ip.cacc, (T)fabs(sg));
      flip = ip.well ? sg > (T)0 : sg < (T)0;
    } else {
      comp_kick<P>(p, ip, pid, l, j, xe.c[0], t, z, kap, sg, fac, flip);
    }
    emit = p.strategy == 1 ? (u3 < fac) : (fac > (T)0);
    if (emit) {
      if (flip) kap = -kap;  // orient by sign(V_W)
      kp.c[0] = P::add(k.c[0], kap);
      km.c[0] = P::sub(k.c[0], kap);
    }
  } else {
    emit = Draw<P>::event4(p, ip, pid, l, j, xe, st, comp, kap, fac, gap);
    if (emit) {
      if (comp != 1) {
        kp.c[0] = P::add(k.c[0], kap);
        km.c[0] = P::sub(k.c[0], kap);
      }
      if (comp == 1) {
        kp.c[1] = P::add(k.c[1], kap);
        km.c[1] = P::sub(k.c[1], kap);
      } else if (comp == 2) {
        kp.c[1] = P::sub(k.c[1], kap);
        km.c[1] = P::add(k.c[1], kap);
      }
    }
  }
  if (emit) {
    static_cast<TanOf<P>&>(b) = tau;
    b.pid = pid;
    b.xe = xe;
    b.kp = kp;
    b.km = km;
    b.t = t;
    b.w = w;
    b.fac = fac;
    b.kap = kap;
    b.l = ent_pack(l, inst);
    b.j = j;
    b.comp = comp;
  }
  return emit;
}

// The pair of an accepted event (Alg. 1 item 3): ids, kills outside the
// k-range, tallies, the event log, then each offspring settled or, when it
// has an event of its own in the interval, handed to `later`.
template <class P, int DST, class Later>
__device__ __forceinline__ void event_pair(const KP<P>& p, const Inst<typename P::T>& ip,
                                           WarpCounts& wc, Acc& acc, const Birth<P>& b,
                                           Later later) {
  using T = typename P::T;
  const int l = ent_l(b.l), inst = ent_inst(b.l);
  const uint4 h = philox_ks(p.ks, (uint32_t)b.pid, (uint32_t)(b.pid >> 32), (uint32_t)l,
                            kDrawPids | b.j);
  const unsigned long long pid_p = (1ull << 63) | ((((unsigned long long)h.y << 32) | h.x) >> 1);
  const unsigned long long pid_m = (1ull << 63) | ((((unsigned long long)h.w << 32) | h.z) >> 1);
  const bool kill_p = !k_inside(p, b.kp);
  const bool kill_m = !k_inside(p, b.km);
  const T wc_ = (P::D == 1 && p.strategy != 1) ? P::mul(b.w, b.fac) : b.w;
  // tangent mode: the birth's score g = (1/H, 1/w - 4 w kappa^2), the
  // derivative of log V_W^+(x_e, kappa) (Eq. 2); the + child gets
  // tau + s g, the - child its negative
  TanOf<P> tp;
  if constexpr (P::TG) {
    const T gw = P::sub(ip.gw0, P::mul(P::mul(ip.gw1, b.kap), b.kap));
    tp.th = P::add(b.th, P::mul(b.w, ip.gH));
    tp.tw = P::add(b.tw, P::mul(b.w, gw));
  }
  ++acc.events;
  if (kill_p) { if (wc_ > (T)0) ++acc.kill_p; else if (wc_ < (T)0) ++acc.kill_m; }
  if (kill_m) { if (-wc_ > (T)0) ++acc.kill_p; else if (-wc_ < (T)0) ++acc.kill_m; }
  if (!P::LEAN && p.log) {
    const unsigned long long idx = atomicAdd(&p.cnt->log_len, 1ull);
    if (idx < (unsigned long long)p.log_cap) {
      wbrw_event ev;
      ev.pid = b.pid;
      ev.pid_plus = pid_p;
      ev.pid_minus = pid_m;
      ev.step = (unsigned)l;
      ev.j = b.j;
      ev.t = (double)b.t;
      ev.xe = (double)b.xe.c[0];
      ev.kappa = (double)b.kap;
      ev.factor = (double)b.fac;
      ev.kill_plus = kill_p;
      ev.kill_minus = kill_m;
      ev.xe2 = (double)b.xe.c[P::D - 1];
      ev.comp = b.comp;
      ev.pad = 0;
      p.log[idx] = ev;
    }
  }
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    if (c == 0 ? kill_p : kill_m) continue;
    SEntry<P> ch;
    if constexpr (P::TG) {
      ch.th = c == 0 ? tp.th : -tp.th;
      ch.tw = c == 0 ? tp.tw : -tp.tw;
    }
    ch.pid = c == 0 ? pid_p : pid_m;
    ch.xo = b.xe;
    ch.to = b.t;
    ch.k = c == 0 ? b.kp : b.km;
    ch.w = c == 0 ? wc_ : -wc_;
    ch.l = b.l;
    ch.j = 0;
    ch.t = Draw<P>::first(p, ip, ch.pid, l, b.t, false, ch.st);
    if (ch.t < p.dt) later(ch);
    else settle<P, DST>(p, wc, acc, inst, ch.pid, ch.xo, ch.to, ch.k, ch.w, l, ch, ch.t);
  }
}

// Event j of a segment at time t: the decision and, when a pair is made,
// the pair.  Returns the gap to the segment's next event.
template <class P, int DST, class Later>
__device__ __forceinline__ typename P::T do_event(const KP<P>& p,
                                                  const Inst<typename P::T>& ip, int inst,
                                                  WarpCounts& wc, Acc& acc,
                                                  unsigned long long pid, const PV<P>& xo,
                                                  typename P::T to, const PV<P>& k,
                                                  typename P::T w,
                                                  const typename Draw<P>::State& st, int l,
                                                  unsigned j, bool root, typename P::T t,
                                                  Later later, const TanOf<P>& tau) {
  typename P::T gap;
  Birth<P> b;
  if (event_decide<P>(p, ip, inst, pid, xo, to, k, w, st, l, j, root, t, tau, b, gap))
    event_pair<P, DST>(p, ip, wc, acc, b, later);
  return gap;
}

// All remaining events of a deferred segment, recursively (drain).
template <class P, int DST>
__device__ void finish_segment(const KP<P>& p, WarpCounts& wc, Acc& acc, const SEntry<P>& s0) {
  SEntry<P> stack[kStack];
  int sp = 0;
  stack[sp++] = s0;
  while (sp > 0) {
    SEntry<P> s = stack[--sp];
    unsigned j = s.j & ~kRootFlag;
    const int inst = ent_inst(s.l), l = ent_l(s.l);
    const Inst<typename P::T> ip = inst_of(p, inst);
    auto later = [&](const SEntry<P>& ch) {
      if (sp < kStack) stack[sp++] = ch;
      else set_err(p.cnt, ERR_NESTING);
    };
    while (s.t < p.dt) {
      const typename P::T gap = do_event<P, DST>(p, ip, inst, wc, acc, s.pid, s.xo, s.to, s.k,
                                                 s.w, s.st, l, j, (s.j & kRootFlag) != 0u, s.t,
                                                 later, s);
      s.t = P::add(s.t, gap);
      ++j;
    }
    if (!(s.j & kRootFlag)) settle<P, DST>(p, wc, acc, inst, s.pid, s.xo, s.to, s.k, s.w, l, s, s.t);
    else chain_next<P>(p, wc, s);
  }
}

// ---------------------------------------------------------------------------
// The flight kernel.  Warp-centric: a warp carries 32 particles at a time
// and never waits for the other warps of its block.  Every particle goes
// through [ls, L) -- streaming plus the candidate clock -- and ends in the
// sink.  The rare candidate intervals become entries (pid, x at the
// interval's start, k, w, l) of the warp's segment of the candidate queue,
// for k_event.
// ---------------------------------------------------------------------------
// A regenerated coordinate moved by single ulps back into its cell idx if
// rounding left it there (Alg. 3 places every particle inside its cell).
template <class P>
__device__ __forceinline__ typename P::T in_cell(typename P::T v, typename P::T lo,
                                                 typename P::T inv, int idx) {
  using T = typename P::T;
  if (P::flr(P::mul(P::sub(v, lo), inv)) == (T)idx) return v;  // the common case
  for (int it = 0; it < 8 && P::flr(P::mul(P::sub(v, lo), inv)) > (T)idx; ++it) v = P::next_dn(v);
  for (int it = 0; it < 8 && P::flr(P::mul(P::sub(v, lo), inv)) < (T)idx; ++it) v = P::next_up(v);
  return v;
}

// Instance of a slot of the base region: the last instance whose first slot
// is <= slot (empty instances share their start with the next one).
template <class P>
__device__ __forceinline__ int base_instance(const KP<P>& p, unsigned long long slot) {
  if (P::SINGLE || p.ninst <= 1) return 0;
  int lo = 0, hi = p.ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.inst_slot[mid] <= slot) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Append one candidate entry per flagged lane (interval c, the position
// streamed from the lane's interval ls to c) to the warp's segment eq_seg
// of the candidate queue (null when the warp owns none); ecount is the
// segment's count, held in a register by every lane.  Every lane of the
// warp calls it.
template <class P>
__device__ __forceinline__ void append_candidate(const KP<P>& p, unsigned& ecount,
                                                 FEntry<P>* eq_seg, bool has,
                                                 unsigned long long pid, const PV<P>& x,
                                                 const PV<P>& k, typename P::T w, int ls, int c,
                                                 int inst, const TanOf<P>& tau) {
  const int lane = threadIdx.x & 31;
  const unsigned bal = __ballot_sync(kFull, has);
  if (has) {
    const unsigned q = ecount + __popc(bal & ((1u << lane) - 1u));
    if (eq_seg && q < p.eseg) {
      FEntry<P> e;
      static_cast<TanOf<P>&>(e) = tau;
      e.pid = pid;
#pragma unroll
      for (int d = 0; d < P::D; ++d) e.x.c[d] = stream_n<P>(x.c[d], k.c[d], p.dtv, c - ls);
      e.k = k;
      e.w = w;
      e.l = ent_pack(c, inst);
      eq_seg[q] = e;
    } else {
      set_err(p.cnt, ERR_CAP_EQUEUE);
    }
  }
  ecount += __popc(bal);
}

template <class P, int SRC, int DST>
__device__ __forceinline__ void flight_tile(const KP<P>& p, WarpCounts& wc, Acc& acc, bool act,
                                            unsigned long long slot, PV<P> x, const PV<P>& k,
                                            typename P::T w, unsigned long long pid, int ls,
                                            int inst, const TanOf<P>& tau,
                                            uint32_t gbits, unsigned& ecount,
                                            FEntry<P>* eq_seg) {
  using T = typename P::T;
  const int lane = threadIdx.x & 31;
  const unsigned g = global_warp();
  const Inst<T> ip = inst_of(p, inst);
  const int cbase = inst * p.nhi;

  // ---- candidate clock over [ls, L) (Sec. 3.2): which intervals hold an
  // event.  Bit b of mask is interval l0 + b.
  unsigned mask = 0;
  const uint32_t plo = (uint32_t)pid, phi = (uint32_t)(pid >> 32);
  if (act) {
    if constexpr (P::is64) {
      for (int l = ls; l < p.L; ++l) {
        const uint4 r = philox_ks(p.ks, plo, phi, (uint32_t)l, 0u);
        if (u53(r.x, r.y) < ip.p_hi) mask |= 1u << (l - p.l0);
      }
    } else if (ls < p.L) {
      // FP32: the first candidate interval from ls on, a geometric gap from
      // 23 random bits: the regeneration draw's (gbits), or the draw (pid,
      // ls, GAP) otherwise.  (FP32 launches no offspring wave: its offspring
      // take their first candidate interval from their next event time, in
      // settle; an entry of an offspring queue would use bits 32..54 of its
      // random id.)
      uint32_t m;
      if constexpr (SRC == SRC_QUEUE) m = (uint32_t)(pid >> 32) & 0x7FFFFFu;
      else if constexpr (SRC == SRC_ARRAY) m = philox_ks(p.ks, plo, phi, (uint32_t)ls, kDrawGap).x >> 9;
      else m = gbits;
      const int c = ls + geo_gap(m, ip.ilq, p.L - ls);
      if (c < p.L) mask = 1u << (c - p.l0);
    }
    acc.psteps += (unsigned)(p.L - ls);
  }

  // ---- the warp's candidate entries.  Entry j of the warp (lanes in
  // order, intervals in order within a lane) goes to queue slot ecount + j and
  // is written by lane j mod 32, which fetches its owner's state with
  // shuffles: every lane stores, and consecutive entries are adjacent.
  if constexpr (!P::is64) {
    // FP32: at most one entry per lane (the first candidate interval)
    if (__ballot_sync(kFull, mask != 0u))
      append_candidate<P>(p, ecount, eq_seg, mask != 0u, pid, x, k, w, ls,
                          p.l0 + __ffs(mask) - 1, inst, tau);
  } else {
  const unsigned cnt = __popc(mask);
  unsigned inc = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += t;
  }
  const unsigned total = __shfl_sync(kFull, inc, 31);
  if (total) {
    const unsigned excl = inc - cnt;
    for (unsigned j0 = 0; j0 < total; j0 += 32) {
      const unsigned j = j0 + lane;
      int o = 0;  // the owner: the number of lanes whose inclusive count is <= j
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) {
        const unsigned v = __shfl_sync(kFull, inc, o + s - 1);
        if (v <= j) o += s;
      }
      o = min(o, 31);
      unsigned mo = __shfl_sync(kFull, mask, o);
      const unsigned eo = __shfl_sync(kFull, excl, o);
      const int lo_s = __shfl_sync(kFull, ls, o);
      const int io = __shfl_sync(kFull, inst, o);
      const unsigned long long po = __shfl_sync(kFull, pid, o);
      const T wo = __shfl_sync(kFull, w, o);
      PV<P> xo, ko;
#pragma unroll
      for (int d = 0; d < P::D; ++d) {
        xo.c[d] = __shfl_sync(kFull, x.c[d], o);
        ko.c[d] = __shfl_sync(kFull, k.c[d], o);
      }
      TanOf<P> to;
      if constexpr (P::TG) {
        to.th = __shfl_sync(kFull, tau.th, o);
        to.tw = __shfl_sync(kFull, tau.tw, o);
      }
      if (j < total) {
        for (unsigned t = j - eo; t; --t) mo &= mo - 1;  // the (j - eo)-th set bit
        const int l = p.l0 + __ffs(mo) - 1;
        const unsigned long long q = (unsigned long long)ecount + j;
        if (eq_seg && q < p.eseg) {
          FEntry<P> e;
          static_cast<TanOf<P>&>(e) = to;
          e.pid = po;
#pragma unroll
          for (int d = 0; d < P::D; ++d) e.x.c[d] = stream_n<P>(xo.c[d], ko.c[d], p.dtv, l - lo_s);
          e.k = ko;
          e.w = wo;
          e.l = ent_pack(l, io);
          eq_seg[q] = e;
        } else {
          set_err(p.cnt, ERR_CAP_EQUEUE);
        }
      }
    }
    ecount += total;
  }
  }

  // ---- free streaming x <- x + (hbar/m) k dt to the end of the period
  if (act) {
#pragma unroll
    for (int d = 0; d < P::D; ++d) x.c[d] = stream_n<P>(x.c[d], k.c[d], p.dtv, p.L - ls);
  }

  // ---- the particle's own final state ----------------------------------
  if constexpr (DST == DST_ARRAY) {
    if constexpr (SRC == SRC_ARRAY) {
      if (act) {
#pragma unroll
        for (int d = 0; d < P::D; ++d) p.x[d * p.capacity + slot] = x.c[d];
      }
    } else if constexpr (SRC == SRC_REGEN && P::TG) {
      // the base region: the signed particles, with tau = 0
      if (act && slot >= (unsigned long long)p.capacity) {
        set_err(p.cnt, ERR_CAP_PARTICLES);
      } else if (act) {
        p.x[slot] = x.c[0];
        p.k[slot] = k.c[0];
        p.s[slot] = w > (T)0 ? 1 : -1;
        p.tan[slot] = 0.0;
        p.tan[p.capacity + slot] = 0.0;
      }
    } else if constexpr (SRC == SRC_REGEN) {
      if (act && slot >= (unsigned long long)p.capacity) {
        set_err(p.cnt, ERR_CAP_PARTICLES);
      } else if (act) {
#pragma unroll
        for (int d = 0; d < P::D; ++d) {
          p.x[d * p.capacity + slot] = x.c[d];
          p.k[d * p.capacity + slot] = k.c[d];
        }
        p.s[slot] = w > (T)0 ? 1 : -1;
        if (p.w) p.w[slot] = w;
      }
    } else {
      const unsigned bal = __ballot_sync(kFull, act);
      unsigned long long off = 0;
      if (lane == 0 && bal) off = atomicAdd(&p.cnt->n, (unsigned long long)__popc(bal));
      off = __shfl_sync(kFull, off, 0) + __popc(bal & ((1u << lane) - 1u));
      if (act) {
        if (off >= (unsigned long long)p.capacity) {
          set_err(p.cnt, ERR_CAP_PARTICLES);
        } else {
#pragma unroll
          for (int d = 0; d < P::D; ++d) {
            p.x[d * p.capacity + off] = x.c[d];
            p.k[d * p.capacity + off] = k.c[d];
          }
          p.s[off] = w > (T)0 ? 1 : (w < (T)0 ? -1 : 0);
          if (p.w) p.w[off] = w;
          if constexpr (P::TG) {
            p.tan[off] = tau.th;
            p.tan[p.capacity + off] = tau.tw;
          }
          p.cpid[off - p.cnt->n_base] = pid;
          if (!P::SINGLE && p.ninst > 1) p.cinst[off - p.cnt->n_base] = (unsigned)inst;
        }
      }
    }
  } else if constexpr (DST == DST_BIN1) {
    // lanes that hit the same cell with the same sign add once (the key is
    // 2 cell + sign, or ~0 for none; 2 nx nk < 2^32 is checked on the host)
    unsigned key = ~0u;
    int cell = -1;
    if (act) {
      if (cell_of<P>(p, x, k, cell)) {
        if (!P::TG || w != (T)0) key = 2u * (unsigned)(cbase + cell) + (w > (T)0 ? 1u : 0u);
      } else {
        cell = -1;
        tally_out<P>(p, acc, w, x, k);
      }
    }
    const unsigned grp = __match_any_sync(kFull, key);
    if (key != ~0u && lane == __ffs(grp) - 1)
      atomicAdd(p.grid + (key >> 1), (key & 1u) ? __popc(grp) : -__popc(grp));
    if constexpr (P::TG) {
      if (act && cell >= 0) add_tangent<P>(p, (long long)cbase + cell, tau);
    }
  } else if constexpr (DST == DST_WSUM) {
    if constexpr (SRC == SRC_REGEN) {
      // regenerated weights are +-1: lanes with the same cell and sign add
      // once, +-(their count) 2^31 (the same fixed-point sum, exactly)
      unsigned key = ~0u;
      if (act) {
        int cell;
        if (cell_of<P>(p, x, k, cell)) key = 2u * (unsigned)(cbase + cell) + (w > (T)0 ? 1u : 0u);
        else tally_out<P>(p, acc, w, x, k);
      }
      const unsigned grp = __match_any_sync(kFull, key);
      if (key != ~0u && lane == __ffs(grp) - 1) {
        const long long v = (long long)__popc(grp) * 2147483648ll;
        atomicAdd((unsigned long long*)(p.wsum + (key >> 1)),
                  (unsigned long long)((key & 1u) ? v : -v));
      }
    } else if (act) {
      int cell;
      if (cell_of<P>(p, x, k, cell))
        atomicAdd((unsigned long long*)(p.wsum + cbase + cell),
                  (unsigned long long)wsum_units<P>(w));
      else tally_out<P>(p, acc, w, x, k);
    }
  } else if constexpr (SRC == SRC_REGEN) {
    // DST_BIN2, regenerated particles: weight +-1, so every one has the same
    // share q = 2^31 N/W of its side (Alg. 2); they are counted per side and
    // cell instead of recorded (lanes with the same cell and side add once),
    // and the bootstrap adds count x (that share's floor and residual) to
    // the cell, the same integer sums as one record each
    unsigned key = ~0u;
    if (act) {
      int cell;
      if (cell_of<P>(p, x, k, cell)) {
        const bool neg = w < (T)0;
        key = 2u * (unsigned)(cbase + cell) + (neg ? 1u : 0u);
        if (!neg) { ++acc.n_plus; acc.w_plus += 2147483648ull; }
        else { ++acc.n_minus; acc.w_minus += 2147483648ull; }
      } else {
        tally_out<P>(p, acc, w, x, k);
      }
    }
    const unsigned grp = __match_any_sync(kFull, key);
    if (key != ~0u && lane == __ffs(grp) - 1)
      atomicAdd(p.ucnt + (size_t)(key & 1u) * ((size_t)p.nhi * p.ninst) + (key >> 1),
                __popc(grp));
  } else {  // DST_BIN2: one record per in-grid particle of nonzero weight
    int cell = -1;
    if (act) {
      if (!cell_of<P>(p, x, k, cell)) { cell = -1; tally_out<P>(p, acc, w, x, k); }
      else if (w == (T)0) cell = -1;
    }
    const unsigned bal = __ballot_sync(kFull, cell >= 0);
    if (bal) {
      const unsigned off = wc.r + __popc(bal & ((1u << lane) - 1u));
      if (cell >= 0) {
        if (g >= (unsigned)p.nseg || off >= p.rseg)
          set_err(p.cnt, ERR_CAP_RECORDS);
        else
          put_record<P>(p, acc, (long long)g * p.rseg + (long long)off, cbase + cell, w);
      }
      __syncwarp();
      if (lane == 0) wc.r += __popc(bal);
      __syncwarp();
    }
  }

}

// The work of one flight launch for the calling warp: its share of the
// source's particles carried through [ls, L) into the sink, their candidate
// intervals appended to the warp's candidate segment (ecount entries so far).
template <class P, int SRC, int DST>
__device__ __forceinline__ void flight_body(const KP<P>& p, WarpCounts& wc, Acc& acc,
                                            unsigned& ecount, FEntry<P>* const eq_seg) {
  using T = typename P::T;
  const int lane = threadIdx.x & 31;
  const unsigned g = global_warp();
  const unsigned long long nwarps = (unsigned long long)gridDim.x * kWarps;

  if constexpr (SRC == SRC_QUEUE) {
    // the previous wave's offspring, one producer segment at a time
    // (the next tile's entries load while the current tile is processed)
    FEntry<P> none{};
    none.l = p.L;
    for (unsigned long long sg = g; sg < (unsigned)p.nseg; sg += nwarps) {
      const unsigned n = min(p.fcnt_in[sg], (unsigned)p.qseg);
      const FEntry<P>* seg = p.fq_in + (long long)sg * p.qseg;
      FEntry<P> nx = (unsigned)lane < n ? seg[lane] : none;
      FEntry<P> nx2 = (unsigned)lane + 32u < n ? seg[lane + 32] : none;
      for (unsigned b = 0; b < n; b += 32) {
        const unsigned i = b + lane;
        const bool act = i < n;
        const FEntry<P> e = nx;
        nx = nx2;
        nx2 = i + 64 < n ? seg[i + 64] : none;
        flight_tile<P, SRC, DST>(p, wc, acc, act, 0, e.x, e.k, e.w, e.pid, ent_l(e.l),
                                 ent_inst(e.l), e, 0u, ecount, eq_seg);
      }
    }
  } else {
    // SRC_TREGEN walks the tangent plan exactly as SRC_REGEN walks the plan
    // of the signed particles
    constexpr bool TR = SRC == SRC_TREGEN;
    constexpr bool RG = SRC == SRC_REGEN || TR;
    const uint32_t* tile_nz = TR ? p.ttile_nz : p.tile_nz;
    const uint32_t* nz_cell = TR ? p.tnz_cell : p.nz_cell;
    const unsigned long long* nz_start = TR ? p.tnz_start : p.nz_start;
    const unsigned long long* islot = TR ? p.tinst_slot : p.inst_slot;
    unsigned long long n;
    if constexpr (SRC == SRC_ARRAY) n = p.cnt->n_src;
    else n = min(TR ? p.cnt->tan_total : p.cnt->regen_total, (unsigned long long)p.tile_cap * 32ull);
    const unsigned long long n_base = p.cnt->n_base, base_pid = p.cnt->base_pid;
    // slots and plan positions of a regeneration index in 32 bits (the
    // capacity is below 2^32 - 2^20, so no sum below overflows)
    using IX = std::conditional_t<RG, unsigned, unsigned long long>;
    const IX nn = (IX)n;
    const IX nz = RG ? (IX)(TR ? p.cnt->tan_nz : p.cnt->nz_count) : (IX)0;
    // regeneration plan entries, loaded ahead: the first nonzero cell a0 two
    // tiles ahead, the starts and cells one tile ahead
    const IX stride = (IX)(nwarps * 32ull);
    IX a0_next = 0, idx_n = 0, st_n = (IX)~0ull;
    uint32_t cw_n = 0u;
    if constexpr (RG) {
      const IX b0 = (IX)(g * 32ull);
      if (b0 < nn) {
        idx_n = tile_nz[b0 >> 5] + lane;
        st_n = idx_n < nz ? (IX)nz_start[idx_n] : (IX)~0ull;
        cw_n = idx_n < nz ? nz_cell[idx_n] : 0u;
      }
      if (b0 + stride < nn) a0_next = tile_nz[(b0 + stride) >> 5];
    }
    // one tile of 32 slots; a full tile (every tile but a warp's last) is
    // compiled apart with every lane active, which drops the per-lane
    // activity tests of the whole flight from the common path
    // one instance: a slot's regeneration draw depends on the slot alone, so
    // the draw of the warp's next tile is made while this tile is processed
    constexpr bool PIPE = P::SINGLE && SRC == SRC_REGEN;
    uint4 r_next = make_uint4(0u, 0u, 0u, 0u);
    if constexpr (PIPE) {
      const unsigned long long q0 = p.regen_base | (unsigned long long)((IX)(g * 32ull) + lane);
      r_next = philox_ks(p.ks, (uint32_t)q0, (uint32_t)(q0 >> 32), kStepRegen, 0u);
    }
    auto tile = [&](const IX base, auto full) {
      const IX slot = base + lane;
      const bool act = decltype(full)::value || slot < nn;
      [[maybe_unused]] const uint4 r_pipe = r_next;
      if constexpr (PIPE) {
        const unsigned long long qn = p.regen_base | (unsigned long long)(slot + stride);
        r_next = philox_ks(p.ks, (uint32_t)qn, (uint32_t)(qn >> 32), kStepRegen, 0u);
      }
      PV<P> x, k;
#pragma unroll
      for (int d = 0; d < P::D; ++d) x.c[d] = k.c[d] = (T)0;
      T w = (T)0;
      unsigned long long pid = 0;
      int inst = 0;
      uint32_t gbits = 0;  // FP32: the first gap's random bits (regeneration)
      TanOf<P> tau;
      if constexpr (P::TG) tau.th = tau.tw = 0.0;
      if constexpr (RG) {
        // Alg. 3: the cell of each slot.  The tile's first nonzero cell a0
        // comes from the plan and holds slot base; the 32 slots of a tile lie
        // in at most 32 nonzero cells, whose starts strictly increase.  Lane i
        // marks bit (start of a0 + i) - base when that start falls inside the
        // tile, and slot base + lane lies in cell a0 + (marks at or below lane).
        [[maybe_unused]] const IX idx = idx_n;  // the tangent plan's tau index
        const IX st = st_n;
        const uint32_t cw = cw_n;
        if (base + stride < nn) {
          idx_n = a0_next + lane;
          st_n = idx_n < nz ? (IX)nz_start[idx_n] : (IX)~0ull;
          cw_n = idx_n < nz ? nz_cell[idx_n] : 0u;
        }
        if (base + 2 * stride < nn) a0_next = tile_nz[(base + 2 * stride) >> 5];
        const unsigned mark =
            (lane > 0 && st > base && st - base < (IX)32) ? 1u << (unsigned)(st - base) : 0u;
        const unsigned marks = __reduce_or_sync(kFull, mark);
        const int lo = __popc(marks & ((2u << lane) - 1u));
        const uint32_t cwl = __shfl_sync(kFull, cw, lo);
        if constexpr (TR) {  // the tangent particles of a cell share its tau
          const T th = idx < nz ? (T)p.tnz_tau[2 * idx] : (T)0;
          const T tw = idx < nz ? (T)p.tnz_tau[2 * idx + 1] : (T)0;
          tau.th = __shfl_sync(kFull, th, lo);
          tau.tw = __shfl_sync(kFull, tw, lo);
        }
        if (act) {
          int cell = (int)(cwl & 0x7FFFFFFFu);
          if (!P::SINGLE && p.ninst > 1) {
            // floor(cell / nhi) from one multiply by ceil(2^40 / nhi): the
            // estimate exceeds the quotient by at most one (cell < 2^30), and
            // cell inst_mag < 2^64 (at most 256 instances)
            inst = (int)(((unsigned long long)(unsigned)cell * p.inst_mag) >> 40);
            if ((unsigned)inst * (unsigned)p.nhi > (unsigned)cell) --inst;
            cell -= inst * p.nhi;
          }
          // tangent particles: ids (epoch << 40) | (instance << 32) | 2^31 | j
          const unsigned long long tag = TR ? 0x80000000ull : 0ull;
          pid = p.regen_base | tag | slot;
          if (!P::SINGLE && p.ninst > 1) pid = p.regen_base | ((unsigned long long)inst << 32) | tag | (slot - islot[inst]);
          uint4 r;
          if constexpr (PIPE) r = r_pipe;
          else r = philox_ks(p.ks, (uint32_t)pid, (uint32_t)(pid >> 32), kStepRegen, 0u);
          if constexpr (P::D == 1) {
            int ix = (int)((float)cell * p.inv_nk);  // exact after one correction (cell < 2^24)
            if (p.nh_big) ix = cell / p.nk;
            int ik = cell - ix * p.nk;
            if (ik < 0) { --ix; ik += p.nk; } else if (ik >= p.nk) { ++ix; ik -= p.nk; }
            T ux, uk;
            if constexpr (P::is64) { ux = (T)u53(r.x, r.y); uk = (T)u53(r.z, r.w); }
            else { ux = (T)u24(r.x); uk = (T)u24(r.y); gbits = r.z >> 9; }
            x.c[0] = in_cell<P>(P::add(p.xmin, P::mul(P::add((T)ix, ux), p.dx)), p.xmin, p.inv_dx, ix);
            k.c[0] = in_cell<P>(P::add(p.kmin, P::mul(P::add((T)ik, uk), p.dk)), p.kmin, p.inv_dk, ik);
          } else {
            // cell = ((ix1 nx + ix2) nk + ik1) nk + ik2; x offsets from the
            // draw (pid, REGEN, 0), k offsets from (pid, REGEN, 1) in FP64,
            // all four from the first draw in FP32
            const int ik2 = cell % p.nk, c1 = cell / p.nk;
            const int ik1 = c1 % p.nk, c2 = c1 / p.nk;
            const int ix2 = c2 % p.nx, ix1 = c2 / p.nx;
            T u[4];
            if constexpr (P::is64) {
              const uint4 r2 = philox_ks(p.ks, (uint32_t)pid, (uint32_t)(pid >> 32), kStepRegen, 1u);
              u[0] = u53(r.x, r.y); u[1] = u53(r.z, r.w); u[2] = u53(r2.x, r2.y); u[3] = u53(r2.z, r2.w);
            } else {
              u[0] = u24(r.x); u[1] = u24(r.y); u[2] = u24(r.z); u[3] = u24(r.w);
              gbits = ((r.x & 0xFFu) << 15) | ((r.y & 0xFFu) << 7) | ((r.z & 0xFFu) >> 1);
            }
            x.c[0] = in_cell<P>(P::add(p.xmin, P::mul(P::add((T)ix1, u[0]), p.dx)), p.xmin, p.inv_dx, ix1);
            x.c[P::D - 1] = in_cell<P>(P::add(p.xmin, P::mul(P::add((T)ix2, u[1]), p.dx)), p.xmin, p.inv_dx, ix2);
            k.c[0] = in_cell<P>(P::add(p.kmin, P::mul(P::add((T)ik1, u[2]), p.dk)), p.kmin, p.inv_dk, ik1);
            k.c[P::D - 1] = in_cell<P>(P::add(p.kmin, P::mul(P::add((T)ik2, u[3]), p.dk)), p.kmin, p.inv_dk, ik2);
          }
          w = TR ? (T)0 : ((cwl >> 31) ? (T)-1 : (T)1);
        }
      } else {
        if (act) {
          if constexpr (P::TG) {
            tau.th = p.tan[slot];
            tau.tw = p.tan[p.capacity + slot];
          }
#pragma unroll
          for (int d = 0; d < P::D; ++d) {
            x.c[d] = p.x[d * p.capacity + slot];
            k.c[d] = p.k[d * p.capacity + slot];
          }
          w = p.w ? p.w[slot] : (T)p.s[slot];
          if (slot < n_base) {
            pid = base_pid + slot;
            if (!P::SINGLE && p.ninst > 1) {
              inst = base_instance(p, slot);
              pid = base_pid + ((unsigned long long)inst << 32) + (slot - p.inst_slot[inst]);
            }
          } else {
            pid = p.cpid[slot - n_base];
            if (!P::SINGLE && p.ninst > 1) inst = (int)p.cinst[slot - n_base];
          }
        }
      }
      flight_tile<P, SRC, DST>(p, wc, acc, act, slot, x, k, w, pid, act ? p.l0 : p.L, inst, tau,
                               gbits, ecount, eq_seg);
    };
    for (IX base = (IX)(g * 32ull); base < nn; base += stride) {
      if (base + (IX)32 <= nn) tile(base, std::true_type{});
      else tile(base, std::false_type{});
    }
  }

}

template <class P, int SRC, int DST>
__global__ void __launch_bounds__(kBlock, (max_blocks<P, DST>())) k_flight(const KP<P> p_) {
  const KP<P> p = with_period(p_);
  __shared__ unsigned long long red[kWarps];
  __shared__ WarpCounts s_wc[kWarps];
  const int lane = threadIdx.x & 31;
  WarpCounts& wc = s_wc[threadIdx.x >> 5];
  Acc acc;
  acc.zero();
  load_counts(p, wc, 0);
  const unsigned g = global_warp();
  // the warp's candidate segment and its count, in registers
  unsigned ecount = wc.e;
  FEntry<P>* const eq_seg = g < (unsigned)p.nseg ? p.eq + (long long)g * p.eseg : nullptr;
  flight_body<P, SRC, DST>(p, wc, acc, ecount, eq_seg);
  if (lane == 0) wc.e = ecount;
  store_counts(p, wc, 0, false, true, DST == DST_BIN2);
  block_reduce_add(red, acc.psteps, &p.cnt->ledger[SRC == SRC_QUEUE ? LG_PSTEPS : LG_PSTEPS0]);
  block_reduce_add(red, acc.out_p, &p.cnt->ledger[LG_OUT_P]);
  block_reduce_add(red, acc.out_m, &p.cnt->ledger[LG_OUT_M]);
  if constexpr (DST == DST_BIN2) {
    block_reduce_add(red, acc.n_plus, &p.cnt->boot_n[0]);
    block_reduce_add(red, acc.n_minus, &p.cnt->boot_n[1]);
    block_reduce_add(red, acc.w_plus, &p.cnt->boot_w[0]);
    block_reduce_add(red, acc.w_minus, &p.cnt->boot_w[1]);
  }
}

// ---------------------------------------------------------------------------
// Event kernels.  k_event takes the candidate intervals of the flight (one
// per lane) and performs their first event; k_cont performs one more event
// of each deferred segment of a level; k_drain finishes the last level.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void reduce_event_tallies(unsigned long long* red, const Acc& acc,
                                                     Counters* c, bool bin2) {
  block_reduce_add(red, acc.psteps, &c->ledger[LG_PSTEPS]);  // FP32 offspring flights
  block_reduce_add(red, acc.events, &c->ledger[LG_EVENTS]);
  block_reduce_add(red, acc.kill_p, &c->ledger[LG_KILL_P]);
  block_reduce_add(red, acc.kill_m, &c->ledger[LG_KILL_M]);
  block_reduce_add(red, acc.out_p, &c->ledger[LG_OUT_P]);
  block_reduce_add(red, acc.out_m, &c->ledger[LG_OUT_M]);
  if (bin2) {
    block_reduce_add(red, acc.n_plus, &c->boot_n[0]);
    block_reduce_add(red, acc.n_minus, &c->boot_n[1]);
    block_reduce_add(red, acc.w_plus, &c->boot_w[0]);
    block_reduce_add(red, acc.w_minus, &c->boot_w[1]);
  }
}

// Asynchronous global -> shared copies (cp.async.ca, 8 bytes each), in
// groups: a thread's wait_group N returns once at most its N most recent
// groups are pending; each thread reads only what it copied itself.
__device__ __forceinline__ void cp_async8(void* dst_smem, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
template <class P>
__device__ __forceinline__ void copy_entry_async(FEntry<P>* dst, const FEntry<P>* src) {
  static_assert(sizeof(FEntry<P>) % 8 == 0 && alignof(FEntry<P>) >= 8, "entry words");
#pragma unroll
  for (unsigned w = 0; w < sizeof(FEntry<P>) / 8; ++w)
    cp_async8((char*)dst + 8 * w, (const char*)src + 8 * w);
}

// One round of the event kernel for the calling warp: the first event of
// each candidate interval in seg[0, n) (one per lane), the pairs, and, in the
// kernels that finish them themselves, every deferred segment; the pairs of
// first events are added to first_pairs.  stage and buf are the warp's
// shared staging tiles and accepted-event buffer.
template <class P, int DST>
__device__ __forceinline__ void event_round(const KP<P>& p, WarpCounts& wc, Acc& acc,
                                            const FEntry<P>* seg, unsigned n,
                                            FEntry<P> (*stage)[32], Birth<P>* buf,
                                            unsigned& first_pairs) {
  using T = typename P::T;
  const int lane = threadIdx.x & 31;
  const unsigned g = global_warp();
  auto later = [&](const SEntry<P>& ch) { defer<P>(p, wc, 1, ch); };
  // FP32 2D: the accepted events of the warp's tiles wait in a per-warp
  // buffer and their pairs are made 32 at a time, so that every lane has one
  // (the acceptance would otherwise leave a third of the lanes idle there);
  // the 4D events, with larger records and more registers, measured slower so
  constexpr bool CMP = !P::is64 && P::D == 1;
  unsigned nb = 0;  // births in the buffer (the same in every lane)
  auto make_pairs = [&](unsigned lim) {
    while (nb >= lim) {
      const unsigned take = min(nb, 32u);
      __syncwarp();
      if ((unsigned)lane < take) {
        const Birth<P> bb = buf[nb - take + lane];
        event_pair<P, DST>(p, inst_of(p, ent_inst(bb.l)), wc, acc, bb, later);
      }
      __syncwarp();
      nb -= take;
    }
  };
  const unsigned events0 = acc.events;
  // each lane copies its entry of the next tile into shared memory
  // asynchronously while the current tile is processed
  if ((unsigned)lane < n) copy_entry_async<P>(&stage[0][lane], seg + lane);
  cp_async_commit();
  unsigned t = 0;
  for (unsigned b = 0; b < n; b += 32, ++t) {
    const unsigned i = b + lane;
    if (i + 32 < n) copy_entry_async<P>(&stage[(t + 1) & 1][lane], seg + i + 32);
    cp_async_commit();
    cp_async_wait<1>();
    FEntry<P> e{};
    if (i < n) e = stage[t & 1][lane];
    bool made = false;
    Birth<P> bb;
    if (i < n) {
      const int l = ent_l(e.l), inst = ent_inst(e.l);
      const Inst<T> ip = inst_of(p, inst);
      SEntry<P> s;
      static_cast<TanOf<P>&>(s) = static_cast<const TanOf<P>&>(e);
      s.pid = e.pid;
      s.xo = e.x;
      s.to = (T)0;
      s.k = e.k;
      s.w = e.w;
      s.l = e.l;
      s.t = Draw<P>::first(p, ip, e.pid, l, (T)0, true, s.st);
      if (s.t < p.dt) {
        ++acc.cand;
        T gap;
        if constexpr (CMP) {
          made = event_decide<P>(p, ip, inst, s.pid, s.xo, s.to, s.k, s.w, s.st, l, 0u, true,
                                 s.t, s, bb, gap);
        } else {
          gap = do_event<P, DST>(p, ip, inst, wc, acc, s.pid, s.xo, s.to, s.k, s.w, s.st, l,
                                 0u, true, s.t, later, s);
        }
        s.t = P::add(s.t, gap);
        if (s.t < p.dt) {
          s.j = 1u | kRootFlag;
          defer<P>(p, wc, 1, s);
        } else {
          chain_next<P>(p, wc, s);
        }
      }
    }
    if constexpr (CMP) {
      const unsigned bal = __ballot_sync(kFull, made);
      if (made) buf[nb + __popc(bal & ((1u << lane) - 1u))] = bb;
      nb += __popc(bal);
      make_pairs(32u);
    }
  }
  cp_async_wait<0>();
  if constexpr (CMP) make_pairs(1u);
  // so far the warp has made only first events' pairs
  first_pairs += acc.events - events0;
  if constexpr (inline_drain<P>()) {
    // These kernels finish their warp's deferred segments here instead of
    // in launches of their own: one event per lane per pass (Alg. 1 item 3,
    // offspring born inside the interval included), a segment with another
    // event in its interval appended again to the same list, until the list
    // is used up.  Its count is then zero for the launches that follow.
    const SEntry<P>* dl = p.dq[1] + (size_t)g * p.dseg;
    unsigned rd = 0;
    for (;;) {
      __syncwarp();
      const unsigned end = min(wc.d, p.dseg);
      if (rd >= end || g >= (unsigned)p.nseg) break;
      const unsigned i = rd + lane;
      if (i < end) {
        SEntry<P> s = dl[i];
        const unsigned j = s.j & ~kRootFlag;
        const int l = ent_l(s.l), inst = ent_inst(s.l);
        const Inst<T> ip = inst_of(p, inst);
        const T gap = do_event<P, DST>(p, ip, inst, wc, acc, s.pid, s.xo, s.to, s.k, s.w, s.st,
                                       l, j, (s.j & kRootFlag) != 0u, s.t, later, s);
        s.t = P::add(s.t, gap);
        if (s.t < p.dt) {
          s.j = (j + 1) | (s.j & kRootFlag);
          defer<P>(p, wc, 1, s);
        } else if (!(s.j & kRootFlag)) {
          settle<P, DST>(p, wc, acc, inst, s.pid, s.xo, s.to, s.k, s.w, l, s, s.t);
        } else {
          chain_next<P>(p, wc, s);
        }
      }
      rd = min(rd + 32u, end);
    }
    __syncwarp();
    if (lane == 0) wc.d = 0;
    __syncwarp();
  }
}

template <class P, int DST>
__global__ void __launch_bounds__(kBlock, (max_blocks<P, DST>())) k_event(const KP<P> p_) {
  const KP<P> p = with_period(p_);
  using T = typename P::T;
  __shared__ unsigned long long red[kWarps];
  __shared__ WarpCounts s_wc[kWarps];
  const int lane = threadIdx.x & 31;
  WarpCounts& wc = s_wc[threadIdx.x >> 5];
  Acc acc;
  acc.zero();
  const unsigned g = global_warp();
  const unsigned long long nwarps = (unsigned long long)gridDim.x * kWarps;
  // a block with no candidate in any of its warps' segments leaves at once
  // (the late rounds of a period hold few): it would append nothing, and its
  // tallies and queue counts would stay as they are
  bool any = false;
  for (unsigned long long sg = g; sg < (unsigned)p.nseg; sg += nwarps) any |= p.ecnt_in[sg] != 0u;
  if (!__syncthreads_or(any)) return;
  load_counts(p, wc, 1);
  auto later = [&](const SEntry<P>& ch) { defer<P>(p, wc, 1, ch); };
  // FP32 2D: the accepted events of the warp's tiles wait in a per-warp
  // buffer and their pairs are made 32 at a time, so that every lane has one
  // (the acceptance would otherwise leave a third of the lanes idle there);
  // the 4D events, with larger records and more registers, measured slower so
  constexpr bool CMP = !P::is64 && P::D == 1;
  constexpr unsigned kBirths = 64;
  __shared__ Birth<P> s_birth[CMP ? kWarps : 1][CMP ? kBirths : 1];
  Birth<P>* buf = s_birth[CMP ? (threadIdx.x >> 5) : 0];
  unsigned nb = 0;  // births in the buffer (the same in every lane)
  __shared__ __align__(16) FEntry<P> s_stage[kWarps][2][32];
  static_assert(sizeof(s_birth) + sizeof(s_stage) + sizeof(s_wc) + sizeof(red) <= 48 * 1024,
                "a block declares at most 48 KB of static shared memory");
  FEntry<P>(*stage)[32] = s_stage[threadIdx.x >> 5];
  auto make_pairs = [&](unsigned lim) {
    while (nb >= lim) {
      const unsigned take = min(nb, 32u);
      __syncwarp();
      if ((unsigned)lane < take) {
        const Birth<P> bb = buf[nb - take + lane];
        event_pair<P, DST>(p, inst_of(p, ent_inst(bb.l)), wc, acc, bb, later);
      }
      __syncwarp();
      nb -= take;
    }
  };
  for (unsigned long long sg = g; sg < (unsigned)p.nseg; sg += nwarps) {
    const unsigned n = min(p.ecnt_in[sg], (unsigned)p.eseg);
    const FEntry<P>* seg = p.eq_in + (long long)sg * p.eseg;
    // each lane copies its entry of the next tile into shared memory
    // asynchronously while the current tile is processed
    if ((unsigned)lane < n) copy_entry_async<P>(&stage[0][lane], seg + lane);
    cp_async_commit();
    unsigned t = 0;
    for (unsigned b = 0; b < n; b += 32, ++t) {
      const unsigned i = b + lane;
      if (i + 32 < n) copy_entry_async<P>(&stage[(t + 1) & 1][lane], seg + i + 32);
      cp_async_commit();
      cp_async_wait<1>();
      FEntry<P> e{};
      if (i < n) e = stage[t & 1][lane];
      bool made = false;
      Birth<P> bb;
      if (i < n) {
        const int l = ent_l(e.l), inst = ent_inst(e.l);
        const Inst<T> ip = inst_of(p, inst);
        SEntry<P> s;
        static_cast<TanOf<P>&>(s) = static_cast<const TanOf<P>&>(e);
        s.pid = e.pid;
        s.xo = e.x;
        s.to = (T)0;
        s.k = e.k;
        s.w = e.w;
        s.l = e.l;
        s.t = Draw<P>::first(p, ip, e.pid, l, (T)0, true, s.st);
        if (s.t < p.dt) {
          ++acc.cand;
          T gap;
          if constexpr (CMP) {
            made = event_decide<P>(p, ip, inst, s.pid, s.xo, s.to, s.k, s.w, s.st, l, 0u, true,
                                   s.t, s, bb, gap);
          } else {
            gap = do_event<P, DST>(p, ip, inst, wc, acc, s.pid, s.xo, s.to, s.k, s.w, s.st, l,
                                   0u, true, s.t, later, s);
          }
          s.t = P::add(s.t, gap);
          if (s.t < p.dt) {
            s.j = 1u | kRootFlag;
            defer<P>(p, wc, 1, s);
          } else {
            chain_next<P>(p, wc, s);
          }
        }
      }
      if constexpr (CMP) {
        const unsigned bal = __ballot_sync(kFull, made);
        if (made) buf[nb + __popc(bal & ((1u << lane) - 1u))] = bb;
        nb += __popc(bal);
        make_pairs(32u);
      }
    }
    cp_async_wait<0>();
  }
  if constexpr (CMP) make_pairs(1u);
  // so far the warp has made only first events' pairs
  const unsigned first_pairs = acc.events;
  if constexpr (inline_drain<P>()) {
    // These kernels finish their warp's deferred segments here instead of
    // in launches of their own: one event per lane per pass (Alg. 1 item 3,
    // offspring born inside the interval included), a segment with another
    // event in its interval appended again to the same list, until the list
    // is used up.  Its count is then zero for the launches that follow.
    const SEntry<P>* dl = p.dq[1] + (size_t)g * p.dseg;
    unsigned rd = 0;
    for (;;) {
      __syncwarp();
      const unsigned end = min(wc.d, p.dseg);
      if (rd >= end || g >= (unsigned)p.nseg) break;
      const unsigned i = rd + lane;
      if (i < end) {
        SEntry<P> s = dl[i];
        const unsigned j = s.j & ~kRootFlag;
        const int l = ent_l(s.l), inst = ent_inst(s.l);
        const Inst<T> ip = inst_of(p, inst);
        const T gap = do_event<P, DST>(p, ip, inst, wc, acc, s.pid, s.xo, s.to, s.k, s.w, s.st,
                                       l, j, (s.j & kRootFlag) != 0u, s.t, later, s);
        s.t = P::add(s.t, gap);
        if (s.t < p.dt) {
          s.j = (j + 1) | (s.j & kRootFlag);
          defer<P>(p, wc, 1, s);
        } else if (!(s.j & kRootFlag)) {
          settle<P, DST>(p, wc, acc, inst, s.pid, s.xo, s.to, s.k, s.w, l, s, s.t);
        } else {
          chain_next<P>(p, wc, s);
        }
      }
      rd = min(rd + 32u, end);
    }
    __syncwarp();
    if (lane == 0) wc.d = 0;
    __syncwarp();
  }
  store_counts(p, wc, 1, true, true, DST == DST_BIN2);
  // the first event of each candidate interval comes before the deferred
  // segments (later events and the offspring's own), so the pairs made up to
  // there are the first events' pairs
  block_reduce_add(red, acc.cand, &p.cnt->ledger[LG_CAND]);
  block_reduce_add(red, first_pairs, &p.cnt->ledger[LG_PAIRS0]);
  reduce_event_tallies(red, acc, p.cnt, DST == DST_BIN2);
}

// A whole resampling period in one launch (the lean models): each warp
// runs its share of the first wave (in the tangent mode, then its share of
// the tangent particles' first wave), then the event rounds over its own
// candidate segments.  Warp g writes candidate segment g and only warp g
// reads it, in this launch as in the launch-per-round schedule, so the
// rounds need no barrier between warps: a warp starts its next round as
// soon as it has finished the previous one, and the warps of an SM mix the
// two phases.  Round r appends to the candidate buffer round r reads not
// (p.eq and p.eq_alt alternate); the deferred segments are finished inside
// each round.  Results are those of the launch-per-round schedule, bit for
// bit (every draw is keyed by particle and interval).
template <class P, int DST>
__global__ void __launch_bounds__(kBlock, 3) k_period(const KP<P> p_) {
  const KP<P> p = with_period(p_);
  __shared__ unsigned long long red[kWarps];
  __shared__ WarpCounts s_wc[kWarps];
  const int lane = threadIdx.x & 31;
  WarpCounts& wc = s_wc[threadIdx.x >> 5];
  Acc acc;
  acc.zero();
  load_counts(p, wc, 1);
  const unsigned g = global_warp();
  const bool own = g < (unsigned)p.nseg;
  // the first wave: candidate intervals into buffer p.eq, segment g
  unsigned ecount = wc.e;
  flight_body<P, SRC_REGEN, DST>(p, wc, acc, ecount, own ? p.eq + (long long)g * p.eseg : nullptr);
  if constexpr (P::TG) {  // the tangent particles of the same histogram join the first wave
    flight_body<P, SRC_TREGEN, DST>(p, wc, acc, ecount,
                                    own ? p.eq + (long long)g * p.eseg : nullptr);
  }
  const unsigned psteps_first = acc.psteps;
  constexpr bool CMP = !P::is64 && P::D == 1;
  constexpr unsigned kBirths = 64;
  __shared__ Birth<P> s_birth[CMP ? kWarps : 1][CMP ? kBirths : 1];
  __shared__ __align__(16) FEntry<P> s_stage[kWarps][2][32];
  static_assert(sizeof(s_birth) + sizeof(s_stage) + sizeof(s_wc) + sizeof(red) <= 48 * 1024,
                "a block declares at most 48 KB of static shared memory");
  unsigned first_pairs = 0;
  unsigned n = own ? min(ecount, p.eseg) : 0u;
  for (int r = 0; r < p.len && n > 0u; ++r) {
    __syncwarp();
    if (lane == 0) {
      wc.e = 0;
      wc.flip = (unsigned)(r + 1) & 1u;  // round r reads buffer r & 1, appends to the other
    }
    __syncwarp();
    event_round<P, DST>(p, wc, acc, ((r & 1) ? p.eq_alt : p.eq) + (long long)g * p.eseg, n,
                        s_stage[threadIdx.x >> 5], s_birth[CMP ? (threadIdx.x >> 5) : 0],
                        first_pairs);
    __syncwarp();
    n = min(wc.e, p.eseg);
  }
  store_counts(p, wc, 1, false, false, DST == DST_BIN2);
  block_reduce_add(red, psteps_first, &p.cnt->ledger[LG_PSTEPS0]);
  block_reduce_add(red, acc.cand, &p.cnt->ledger[LG_CAND]);
  block_reduce_add(red, first_pairs, &p.cnt->ledger[LG_PAIRS0]);
  acc.psteps -= psteps_first;  // the offspring's flights
  reduce_event_tallies(red, acc, p.cnt, DST == DST_BIN2);
}

template <class P, int DST>
__global__ void __launch_bounds__(kBlock, (max_blocks<P, DST>())) k_cont(const KP<P> p_, int level) {
  const KP<P> p = with_period(p_);
  using T = typename P::T;
  __shared__ unsigned long long red[kWarps];
  __shared__ WarpCounts s_wc[kWarps];
  const int lane = threadIdx.x & 31;
  WarpCounts& wc = s_wc[threadIdx.x >> 5];
  Acc acc;
  acc.zero();
  const unsigned g = global_warp();
  const unsigned long long nwarps = (unsigned long long)gridDim.x * kWarps;
  const SEntry<P>* in = ((level & 1) ? p.dq[1] : p.dq[0]);
  const unsigned* in_cnt = p.dcnt + (long long)level * p.nseg;
  bool any = false;  // a block with nothing to do leaves at once
  for (unsigned long long sg = g; sg < (unsigned)p.nseg; sg += nwarps) any |= in_cnt[sg] != 0u;
  if (!__syncthreads_or(any)) return;
  load_counts(p, wc, level + 1);
  auto later = [&](const SEntry<P>& ch) { defer<P>(p, wc, level + 1, ch); };
  for (unsigned long long sg = g; sg < (unsigned)p.nseg; sg += nwarps) {
    const unsigned n = min(in_cnt[sg], (unsigned)p.dseg);
    for (unsigned b = 0; b < n; b += 32) {
      const unsigned i = b + lane;
      if (i < n) {
        SEntry<P> s = in[(long long)sg * p.dseg + i];
        const unsigned j = s.j & ~kRootFlag;
        const int l = ent_l(s.l), inst = ent_inst(s.l);
        const Inst<T> ip = inst_of(p, inst);
        const T gap = do_event<P, DST>(p, ip, inst, wc, acc, s.pid, s.xo, s.to, s.k, s.w, s.st,
                                       l, j, (s.j & kRootFlag) != 0u, s.t, later, s);
        s.t = P::add(s.t, gap);
        if (s.t < p.dt) {
          s.j = (j + 1) | (s.j & kRootFlag);
          defer<P>(p, wc, level + 1, s);
        } else if (!(s.j & kRootFlag)) {
          settle<P, DST>(p, wc, acc, inst, s.pid, s.xo, s.to, s.k, s.w, l, s, s.t);
        } else {
          chain_next<P>(p, wc, s);
        }
      }
    }
  }
  store_counts(p, wc, level + 1, true, true, DST == DST_BIN2);
  reduce_event_tallies(red, acc, p.cnt, DST == DST_BIN2);
}

template <class P, int DST>
__global__ void __launch_bounds__(kBlock, (max_blocks<P, DST>())) k_drain(const KP<P> p_, int level) {
  const KP<P> p = with_period(p_);
  __shared__ unsigned long long red[kWarps];
  __shared__ WarpCounts s_wc[kWarps];
  const int lane = threadIdx.x & 31;
  WarpCounts& wc = s_wc[threadIdx.x >> 5];
  Acc acc;
  acc.zero();
  const unsigned g = global_warp();
  const unsigned long long nwarps = (unsigned long long)gridDim.x * kWarps;
  const SEntry<P>* in = ((level & 1) ? p.dq[1] : p.dq[0]);
  const unsigned* in_cnt = p.dcnt + (long long)level * p.nseg;
  bool any = false;  // a block with nothing to do leaves at once
  for (unsigned long long sg = g; sg < (unsigned)p.nseg; sg += nwarps) any |= in_cnt[sg] != 0u;
  if (!__syncthreads_or(any)) return;
  load_counts(p, wc, 0);
  for (unsigned long long sg = g; sg < (unsigned)p.nseg; sg += nwarps) {
    const unsigned n = min(in_cnt[sg], (unsigned)p.dseg);
    for (unsigned i = lane; i < n; i += 32)
      finish_segment<P, DST>(p, wc, acc, in[(long long)sg * p.dseg + i]);
  }
  store_counts(p, wc, 0, true, true, DST == DST_BIN2);
  reduce_event_tallies(red, acc, p.cnt, DST == DST_BIN2);
}

// Initial particles from the Gaussian-wavepacket Wigner function (positive):
// Box-Muller on the init stream of pid = (instance << 32) | index, with
// x ~ N(x0, sx^2), k ~ N(k0, sk^2) of the slot's instance.
template <class P>
__global__ void __launch_bounds__(kBlock) k_init(const KP<P> p, const InitInst* ini,
                                                 unsigned long long n) {
  using T = typename P::T;
  for (unsigned long long i = (unsigned long long)blockIdx.x * kBlock + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * kBlock) {
    const int inst = base_instance(p, i);
    const InitInst g = ini[inst];
    const unsigned long long pid = ((unsigned long long)inst << 32) | (i - g.start);
    const uint4 r = philox_ks(p.ks, (uint32_t)pid, (uint32_t)(pid >> 32), kStepInit, 0u);
#pragma unroll
    for (int e = 0; e < P::D; ++e) {  // electron e of the 4D model: its own pair of draws
      const double x0 = e == 0 ? g.x0 : g.x0b, k0 = e == 0 ? g.k0 : g.k0b;
      T x, k;
      if constexpr (P::is64) {
        const uint4 q =
            e == 0 ? r : philox_ks(p.ks, (uint32_t)pid, (uint32_t)(pid >> 32), kStepInit, (uint32_t)e);
        const double ua = u53(q.x, q.y), ub = u53(q.z, q.w);
        const double rad = __dsqrt_rn(__dmul_rn(-2.0, log1p(-ua)));
        const double th = __dmul_rn(6.283185307179586476925286766559, ub);
        x = (T)__dadd_rn(x0, __dmul_rn(g.sx, __dmul_rn(rad, cos(th))));
        k = (T)__dadd_rn(k0, __dmul_rn(g.sk, __dmul_rn(rad, sin(th))));
      } else {
        const float ua = u24(e == 0 ? r.x : r.z), ub = u24(e == 0 ? r.y : r.w);
        const float rad = sqrtf(-2.0f * log1pf(-ua));
        float sn, cs;
        sincospif(2.0f * ub, &sn, &cs);
        x = (T)(x0 + g.sx * (double)(rad * cs));
        k = (T)(k0 + g.sk * (double)(rad * sn));
      }
      p.x[e * p.capacity + i] = x;
      p.k[e * p.capacity + i] = k;
    }
    p.s[i] = 1;
    if (p.w) p.w[i] = (T)1;
  }
}

// Stream ids (and instances, if inst_out is not NULL) of the materialised
// particles.
template <class P>
__global__ void __launch_bounds__(kBlock) k_pids(const KP<P> p, unsigned long long* out,
                                                 unsigned* inst_out) {
  const unsigned long long n = p.cnt->n, nb = p.cnt->n_base, bp = p.cnt->base_pid;
  for (unsigned long long i = (unsigned long long)blockIdx.x * kBlock + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * kBlock) {
    int inst = 0;
    unsigned long long pid;
    if (i < nb) {
      inst = base_instance(p, i);
      pid = bp + ((unsigned long long)inst << 32) + (i - p.inst_slot[inst]);
    } else {
      pid = p.cpid[i - nb];
      if (!P::SINGLE && p.ninst > 1) inst = (int)p.cinst[i - nb];
    }
    if (out) out[i] = pid;
    if (inst_out) inst_out[i] = (unsigned)inst;
  }
}

}  // namespace wbrw

// ---------------------------------------------------------------------------
// Host-side driver of the kernels above for one precision.
// ---------------------------------------------------------------------------
namespace wbrw {

template <class P>
KP<P> make_kp(const Ctx* c) {
  using T = typename P::T;
  KP<P> p{};  // fields a kernel does not use stay zero (null pointers)
  const wbrw_config& g = c->cfg;
  p.dt = (T)g.dt;
  p.inv_dt = (T)(1.0 / g.dt);
  p.dt_lo = std::nextafter((T)g.dt, (T)-1e30);
  p.dtv = (T)c->dtv;
  p.hm = (T)c->hm;
  p.xmin = (T)g.xmin;
  p.kmin = (T)g.kmin;
  p.kmax = (T)g.kmax;
  p.dx = (T)c->dx;
  p.dk = (T)c->dk;
  p.inv_dx = (T)c->inv_dx;
  p.inv_dk = (T)c->inv_dk;
  p.nx = g.nx;
  p.nk = g.nk;
  p.inv_nk = 1.0f / (float)g.nk;
  p.nh_big = (long long)c->nhi >= (1ll << 24);
  p.inst_mag = ((1ull << 40) + (unsigned long long)c->nhi - 1ull) / (unsigned long long)c->nhi;
  p.ninst = c->ninst;
  p.nhi = (int)c->nhi;
  p.inst = (const Inst<T>*)c->inst_tab;
  p.inst0 = *(const Inst<T>*)c->host_tab;
  p.inst_slot = c->inst_slot;
  p.cinst = c->cinst;
  for (int r = 0; r < 10; ++r) {
    p.ks.k0[r] = (uint32_t)g.seed + (uint32_t)r * 0x9E3779B9u;
    p.ks.k1[r] = (uint32_t)(g.seed >> 32) + (uint32_t)r * 0xBB67AE85u;
  }
  p.strategy = g.strategy;
  p.l0 = p.L = (int)c->step;
  p.len = 0;
  for (int t = 0; t < 2; ++t) {
    p.tab.xi[t] = (const T*)c->tab_xi[t];
    p.tab.cdf[t] = (const T*)c->tab_cdf[t];
    p.tab.guide[t] = c->tab_guide[t];
    p.tab.Y[t] = c->tab_Y[t];
    p.tab.inv_dy[t] = c->tab_inv_dy[t];
    p.tab.gam[t] = c->tab_gam[t];
  }
  p.tab.xc = c->pot.xc;
  p.tab.kap0 = (T)(-c->tab_K);
  p.tab.dkap = (T)c->tab_dkap;
  p.tab.ny = c->tab_ny;
  p.tab.nkap = c->tab_nkap;
  p.comp = (const Comp*)c->comp_tab;
  p.ncomp = c->ncomp;
  p.dgrid[0] = c->dgrid[0];
  p.dgrid[1] = c->dgrid[1];
  p.tan = (double*)c->buf.tangent;
  p.tnz_cell = c->tnz_cell;
  p.tnz_start = c->tnz_start;
  p.tnz_tau = c->tnz_tau;
  p.ttile_nz = c->ttile_nz;
  p.tinst_slot = c->tinst_slot;
  p.regen_base = (unsigned long long)c->epoch << 40;
  p.x = (T*)c->buf.x;
  p.k = (T*)c->buf.k;
  p.s = c->buf.s;
  p.w = g.strategy != WBRW_SP1_PAIR ? (T*)c->buf.w : nullptr;  // sp2 and wp
  p.capacity = c->buf.capacity;
  p.cpid = c->cpid;
  p.nseg = c->nseg;
  p.fq_in = (FEntry<P>*)c->fq[0];
  p.fcnt_in = c->fcnt[0];
  p.fq_out = (FEntry<P>*)c->fq[1];
  p.fcnt_out = c->fcnt[1];
  p.qseg = (unsigned)c->qseg;
  p.eq = (FEntry<P>*)c->eq[0];
  p.ecnt = c->ecnt[0];
  p.eq_in = (const FEntry<P>*)c->eq[1];
  p.ecnt_in = c->ecnt[1];
  p.eseg = (unsigned)c->eseg;
  p.dq[0] = (SEntry<P>*)c->dq[0];
  p.dq[1] = (SEntry<P>*)c->dq[1];
  p.dcnt = c->dcnt;
  p.dseg = (unsigned)c->dseg;
  p.rec_cell = c->rec_cell;
  p.rec_a = c->rec_a;
  p.rcnt = c->cfg.strategy == WBRW_SP2_BOOTSTRAP ? c->rcnt : nullptr;
  p.rseg = (unsigned)c->rseg;
  p.ucnt = c->boot_ucnt;
  p.grid = c->buf.grid;
  p.wsum = c->tmp_wsum;
  p.rec_cell = c->rec_cell;
  p.rec_a = c->rec_a;
  p.nz_cell = c->nz_cell;
  p.nz_start = c->nz_start;
  p.tile_nz = c->tile_nz;
  p.tile_cap = c->tile_cap;
  p.cnt = c->cnt;
  p.log = (wbrw_event*)c->buf.event_log;
  p.log_cap = c->buf.event_log ? c->buf.event_log_capacity : 0;
  p.count_ledger = 1;
  return p;
}

// Every queue kernel runs the same number of resident blocks per SM (the
// context's tuning, at most its model's max_blocks): producer warp g owns queue
// segment g and consumer warp g reads it, so equal grids keep the segments
// matched one to one (nseg of them).
template <class K>
int occupancy(K kern) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm;
}

inline int grid_of(const Ctx* c, int occ) {
  const int per_sm = occ < c->bps ? occ : c->bps;
  int g = per_sm * c->num_sms;
  if (g * kWarps > c->nseg) g = c->nseg / kWarps;
  return g;
}

template <class P, int SRC, int DST>
cudaError_t flight(Ctx* c, const KP<P>& p) {
  static const int occ = occupancy(k_flight<P, SRC, DST>);
  k_flight<P, SRC, DST><<<grid_of(c, occ), kBlock, 0, c->stream>>>(p);
  c->launches++;
  return cudaGetLastError();
}

template <class P, int DST>
cudaError_t events(Ctx* c, const KP<P>& p, int r) {
  static const int o_ev = occupancy(k_event<P, DST>);
  static const int o_cont = occupancy(k_cont<P, DST>);
  static const int o_drain = occupancy(k_drain<P, DST>);
  prof_begin(c, PROF_EVENT, r);
  k_event<P, DST><<<grid_of(c, o_ev), kBlock, 0, c->stream>>>(p);
  prof_end(c, PROF_EVENT, r);
  c->launches += 1;
  if constexpr (!inline_drain<P>()) {  // else the event kernel finished every segment itself
    for (int level = 1; level <= c->passes; ++level)
      k_cont<P, DST><<<grid_of(c, o_cont), kBlock, 0, c->stream>>>(p, level);
    k_drain<P, DST><<<grid_of(c, o_drain), kBlock, 0, c->stream>>>(p, c->passes + 1);
    c->launches += c->passes + 1;
  }
  return cudaGetLastError();
}

template <class P, int DST>
cudaError_t flight_src(Ctx* c, const KP<P>& p, int src) {
  if constexpr (P::TG) {
    if (src == SRC_TREGEN) return flight<P, SRC_TREGEN, DST>(c, p);
  }
  switch (src) {
    case SRC_ARRAY: return flight<P, SRC_ARRAY, DST>(c, p);
    case SRC_REGEN: return flight<P, SRC_REGEN, DST>(c, p);
    default: return flight<P, SRC_QUEUE, DST>(c, p);
  }
}

template <class P>
cudaError_t flight_any(Ctx* c, const KP<P>& p, int src, int dst) {
  if (dst == DST_ARRAY) return flight_src<P, DST_ARRAY>(c, p, src);
  if (dst == DST_BIN1) return flight_src<P, DST_BIN1>(c, p, src);
  if constexpr (P::D == 1 && !P::TG) {  // weighted sinks: sp2 and its observables (2D only)
    if (dst == DST_BIN2) return flight_src<P, DST_BIN2>(c, p, src);
    return flight_src<P, DST_WSUM>(c, p, src);
  }
  return cudaErrorNotSupported;
}

template <class P>
cudaError_t events_any(Ctx* c, const KP<P>& p, int dst, int r) {
  if (dst == DST_ARRAY) return events<P, DST_ARRAY>(c, p, r);
  if (dst == DST_BIN1) return events<P, DST_BIN1>(c, p, r);
  if constexpr (P::D == 1 && !P::TG) {
    if (dst == DST_BIN2) return events<P, DST_BIN2>(c, p, r);
    return events<P, DST_WSUM>(c, p, r);
  }
  return cudaErrorNotSupported;
}

// One regenerating period of a lean model in one launch (k_period): the
// candidate and deferred counts start at zero, the first wave's candidates go
// to buffer 0 and the rounds alternate between the two buffers.
template <class P, int DST>
cudaError_t period(Ctx* c, KP<P> p, size_t cnt_bytes) {
  static const int occ = occupancy(k_period<P, DST>);
  cudaError_t e;
  if ((e = launch_zero(c, c->ecnt[0], cnt_bytes)) != cudaSuccess) return e;
  if ((e = launch_zero(c, c->dcnt, (size_t)(c->passes + 2) * cnt_bytes)) != cudaSuccess) return e;
  p.eq = (FEntry<P>*)c->eq[0];
  p.ecnt = c->ecnt[0];
  p.eq_alt = (FEntry<P>*)c->eq[1];
  prof_begin(c);
  k_period<P, DST><<<grid_of(c, occ), kBlock, 0, c->stream>>>(p);
  prof_end(c);
  c->launches++;
  return cudaGetLastError();
}

template <class P>
cudaError_t period_any(Ctx* c, const KP<P>& p, int dst, size_t cnt_bytes) {
  if constexpr (fused_period<P>()) {
    if (dst == DST_BIN1) return period<P, DST_BIN1>(c, p, cnt_bytes);
    // wp's weight sums too (on the 1e8-particle workload 3.97 against 4.72 ms
    // per period); sp2's record sink runs launch per round
    if constexpr (P::D == 1 && !P::TG) {
      if (dst == DST_WSUM) return period<P, DST_WSUM>(c, p, cnt_bytes);
    }
  }
  return cudaErrorNotSupported;
}

// The kernel tables of the 4D model, one thread per row of either type.
// Row i of type t: v_j = max(A_tj sin(2 y_i kappa_j), 0) for the cells j in
// order, y_i = -Y_t + i dy_t, kappa_j = kap0 + (j + 1/2) dkappa; S_j = the
// running sum of v; xi_i = S_last dkappa.  FP64 rows hold S, FP32 rows S/S_last
// (a second pass).  The largest xi of each type goes to xmax[t] (positive
// doubles order like their bit patterns).
template <class T>
__global__ void __launch_bounds__(kBlock) k_tab4(const double* A, int ny, int nkap,
                                                 double Y0, double dy0, double Y1, double dy1,
                                                 double kap0, double dkap, T* cdf0, T* cdf1,
                                                 T* xi0, T* xi1, unsigned long long* xmax) {
  const int row = blockIdx.x * kBlock + threadIdx.x;
  if (row >= 2 * ny) return;
  const int t = row / ny, i = row % ny;
  const double* At = A + (long long)t * nkap;
  const double y = __dadd_rn(-(t ? Y1 : Y0), __dmul_rn((double)i, t ? dy1 : dy0));
  T* out = (t ? cdf1 : cdf0) + (long long)i * nkap;
  double acc = 0.0;
  for (int j = 0; j < nkap; ++j) {
    const double kap = __dadd_rn(kap0, __dmul_rn(__dadd_rn((double)j, 0.5), dkap));
    const double v = __dmul_rn(At[j], sin(__dmul_rn(__dmul_rn(2.0, y), kap)));
    if (v > 0.0) acc = __dadd_rn(acc, v);
    if constexpr (sizeof(T) == 8) out[j] = (T)acc;
  }
  const double xi = __dmul_rn(acc, dkap);
  if constexpr (sizeof(T) == 4) {
    double run = 0.0;
    for (int j = 0; j < nkap; ++j) {
      const double kap = __dadd_rn(kap0, __dmul_rn(__dadd_rn((double)j, 0.5), dkap));
      const double v = __dmul_rn(At[j], sin(__dmul_rn(__dmul_rn(2.0, y), kap)));
      if (v > 0.0) run = __dadd_rn(run, v);
      out[j] = acc > 0.0 ? (T)(run / acc) : (T)0;
    }
  }
  (t ? xi1 : xi0)[i] = (T)xi;
  atomicMax(xmax + t, (unsigned long long)__double_as_longlong(xi));
}

// Guide tables of the FP32 4D kick rows (the indexed search of Chen and
// Asau): entry b < 2^kTabGuideBits of row i is the first cell whose
// normalised cumulative sum exceeds b 2^-kTabGuideBits (nkap - 1 if none),
// entry 2^kTabGuideBits is nkap - 1.  A target u in [b, b + 1) 2^-kTabGuideBits
// has its cell in [G_b, G_(b+1)].
template <class T>
__global__ void __launch_bounds__(kBlock) k_tab4_guide(const T* cdf0, const T* cdf1, int ny,
                                                       int nkap, int* guide0, int* guide1) {
  const long long per = (long long)ny * (kTabGuide + 1);
  for (long long i = (long long)blockIdx.x * kBlock + threadIdx.x; i < 2 * per;
       i += (long long)gridDim.x * kBlock) {
    const int t = i < per ? 0 : 1;
    const long long k = i - t * per;
    const int row = (int)(k / (kTabGuide + 1)), b = (int)(k - (long long)row * (kTabGuide + 1));
    const T* r = (t ? cdf1 : cdf0) + (long long)row * nkap;
    int lo = 0, hi = nkap - 1;
    if (b < kTabGuide) {
      const T thr = (T)b * ((T)1 / (T)kTabGuide);
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (r[mid] > thr) hi = mid; else lo = mid + 1;
      }
    } else {
      lo = nkap - 1;
    }
    (t ? guide1 : guide0)[k] = lo;
  }
}

template <class P>
struct DriverImpl {
  // The per-instance tables (physics, initial sampling, first slots) are
  // staged in c->host_tab and copied to the scratch before the first launch.
  static cudaError_t init(Ctx* c, long long n) {
    using T = typename P::T;
    char* h = (char*)c->host_tab;
    Inst<T>* it = (Inst<T>*)h;
    InitInst* ii = (InitInst*)(h + kInstTabBytes);
    unsigned long long* is = (unsigned long long*)(h + kTabSlotOff);
    double* na = (double*)(h + kTabNaOff);
    for (int i = 0; i < c->ninst; ++i) {
      const InstHost& q = c->ih[i];
      Inst<T> v;
      v.gamma0 = (T)q.gamma0;
      v.cacc = (T)q.cacc;
      v.sig_k = (T)q.sig_k;
      v.xc = (T)q.xc;
      v.well = q.H < 0.0;
      v.gH = q.H != 0.0 ? 1.0 / q.H : 0.0;
      v.gw0 = 1.0 / q.w;
      v.gw1 = 4.0 * q.w;
      v.p_hi = q.p_any * (1.0 + 1e-9) + 1e-300;
      v.p_any_f = (float)q.p_any;
      v.ilq = (float)(1.0 / log1p(-q.p_any));  // -inf for p_any = 0, -0 for p_any = 1
      v.ig0 = q.gamma0 > 0.0 ? (float)(1.0 / q.gamma0) : 0.0f;
      it[i] = v;
      InitInst g;
      g.x0 = q.x0;
      g.sx = q.sx;
      g.k0 = q.k0;
      g.sk = 1.0 / (2.0 * q.sx);
      g.start = q.start;
      g.x0b = q.x0b;
      g.k0b = q.k0b;
      ii[i] = g;
      is[i] = q.start;
      na[i] = (double)q.n_alpha;
    }
    is[c->ninst] = (unsigned long long)n;
    static_assert(sizeof(Inst<double>) <= kInstBytes && sizeof(Inst<float>) <= kInstBytes,
                  "instance record size");
    static_assert(sizeof(InitInst) <= kInstBytes, "instance record size");
    cudaError_t e = cudaMemcpyAsync(c->inst_tab, h, kTabTransOff, cudaMemcpyHostToDevice,
                                    c->stream);
    if (e != cudaSuccess) return e;
    if ((e = launch_setup(c, SETUP_INIT, (unsigned long long)n, 0)) != cudaSuccess) return e;
    KP<P> p = make_kp<P>(c);
    static const int occ = occupancy(k_init<P>);
    k_init<P><<<occ * c->num_sms, kBlock, 0, c->stream>>>(p, (const InitInst*)((char*)c->inst_tab + kInstTabBytes),
                                              (unsigned long long)n);
    c->launches++;
    return cudaGetLastError();
  }

  // Intervals [l0, L): round r carries the particles that start at l0 + r
  // or later; offspring start one interval after their birth, so L - l0
  // rounds drain every wave.
  static cudaError_t chunk(Ctx* c, int l0, int L, int src, int dst) {
    cudaError_t e = launch_setup(c, c->capturing ? SETUP_CHUNK_DEV : SETUP_CHUNK,
                                 (unsigned long long)l0, (unsigned long long)c->epoch << 40);
    if (e != cudaSuccess) return e;
    KP<P> p = make_kp<P>(c);
    p.l0 = l0;
    p.L = L;
    p.len = L - l0;
    const int rounds = L > l0 ? L - l0 : 1;
    const size_t cnt_bytes = (size_t)c->nseg * sizeof(unsigned);
    if constexpr (fused_period<P>()) {
      if (c->one_launch && src == SRC_REGEN && L > l0 && (dst == DST_BIN1 || dst == DST_WSUM))
        return period_any<P>(c, p, dst, cnt_bytes);
    }
    for (int r = 0; r < rounds; ++r) {
      p.fq_in = (FEntry<P>*)c->fq[r & 1];
      p.fcnt_in = c->fcnt[r & 1];
      p.fq_out = (FEntry<P>*)c->fq[(r + 1) & 1];
      p.fcnt_out = c->fcnt[(r + 1) & 1];
      // round r's candidates: those k_event of round r - 1 chained (FP32),
      // then those of the round's flight
      p.eq = (FEntry<P>*)c->eq[r & 1];
      p.ecnt = c->ecnt[r & 1];
      if (r == 0 && (e = launch_zero(c, p.ecnt, cnt_bytes)) != cudaSuccess) return e;
      if (r == 0) prof_begin(c);
      // FP32 offspring fly inside the event kernels that settle them; FP64
      // offspring fly in a wave of their own (the per-interval draws)
      if (r == 0 || P::is64) e = flight_any<P>(c, p, r == 0 ? src : (int)SRC_QUEUE, dst);
      if (r == 0) prof_end(c);
      if (e != cudaSuccess) return e;
      if (P::TG && r == 0 && src == SRC_REGEN) {
        // the tangent particles of the same histogram join the first wave
        // (the same round: they continue the round's queue counts)
        if ((e = flight_any<P>(c, p, SRC_TREGEN, dst)) != cudaSuccess) return e;
      }
      if (L > l0) {
        p.eq_in = p.eq;
        p.ecnt_in = p.ecnt;
        p.eq = (FEntry<P>*)c->eq[(r + 1) & 1];
        p.ecnt = c->ecnt[(r + 1) & 1];
        if ((e = launch_zero(c, p.ecnt, cnt_bytes)) != cudaSuccess) return e;
        if ((e = launch_zero(c, p.fcnt_out, cnt_bytes)) != cudaSuccess) return e;
        if ((e = launch_zero(c, c->dcnt, (size_t)(c->passes + 2) * cnt_bytes)) != cudaSuccess)
          return e;
        e = events_any<P>(c, p, dst, r);
        if (e != cudaSuccess) return e;
      }
    }
    return cudaSuccess;
  }

  static cudaError_t bin(Ctx* c, int dst, int* grid, int count_ledger) {
    cudaError_t e = launch_setup(c, SETUP_CHUNK, (unsigned long long)c->step,
                                 (unsigned long long)c->epoch << 40);
    if (e != cudaSuccess) return e;
    KP<P> p = make_kp<P>(c);
    p.grid = grid;
    p.count_ledger = count_ledger;
    if (!count_ledger) p.dgrid[0] = p.dgrid[1] = nullptr;  // observables only
    return flight_any<P>(c, p, SRC_ARRAY, dst);
  }

  static cudaError_t materialize(Ctx* c) {
    cudaError_t e = launch_setup(c, SETUP_AFTER_REGEN, (unsigned long long)c->epoch << 40,
                                 (unsigned long long)c->step);
    if (e != cudaSuccess) return e;
    KP<P> p = make_kp<P>(c);
    e = flight<P, SRC_REGEN, DST_ARRAY>(c, p);
    if constexpr (P::TG) {  // the tangent particles, appended
      if (e == cudaSuccess) e = flight<P, SRC_TREGEN, DST_ARRAY>(c, p);
    }
    return e;
  }

  // Build the 4D model's tables from A (host, 2 x nkap) into the scratch and
  // return the largest xi of each type.
  static cudaError_t tables(Ctx* c, const double* A_host, double* xmax_host) {
    using T = typename P::T;
    if constexpr (P::D == 2) {
      cudaError_t e = cudaMemcpyAsync(c->tab_A, A_host, (size_t)2 * c->tab_nkap * sizeof(double),
                                      cudaMemcpyHostToDevice, c->stream);
      if (e != cudaSuccess) return e;
      if ((e = cudaMemsetAsync(c->tab_xmax, 0, 2 * sizeof(unsigned long long), c->stream)) !=
          cudaSuccess)
        return e;
      const int nrow = 2 * c->tab_ny;
      k_tab4<T><<<(nrow + kBlock - 1) / kBlock, kBlock, 0, c->stream>>>(
          c->tab_A, c->tab_ny, c->tab_nkap, c->tab_Y[0], c->tab_dy[0], c->tab_Y[1],
          c->tab_dy[1], -c->tab_K, c->tab_dkap, (T*)c->tab_cdf[0], (T*)c->tab_cdf[1],
          (T*)c->tab_xi[0], (T*)c->tab_xi[1], c->tab_xmax);
      c->launches++;
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if constexpr (!P::is64) {
        const long long ng = 2ll * c->tab_ny * (kTabGuide + 1);
        k_tab4_guide<T><<<(unsigned)((ng + kBlock - 1) / kBlock), kBlock, 0, c->stream>>>(
            (const T*)c->tab_cdf[0], (const T*)c->tab_cdf[1], c->tab_ny, c->tab_nkap,
            c->tab_guide[0], c->tab_guide[1]);
        c->launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
      }
      unsigned long long m[2];
      if ((e = cudaMemcpyAsync(m, c->tab_xmax, sizeof(m), cudaMemcpyDeviceToHost, c->stream)) !=
          cudaSuccess)
        return e;
      if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return e;
      for (int t = 0; t < 2; ++t) {
        double v;
        memcpy(&v, &m[t], sizeof(v));
        xmax_host[t] = v;
      }
      return cudaSuccess;
    } else {
      (void)c;
      (void)A_host;
      (void)xmax_host;
      return cudaErrorNotSupported;
    }
  }

  static cudaError_t pids(Ctx* c, unsigned long long* out, unsigned* inst_out) {
    KP<P> p = make_kp<P>(c);
    static const int occ = occupancy(k_pids<P>);
    k_pids<P><<<occ * c->num_sms, kBlock, 0, c->stream>>>(p, out, inst_out);
    c->launches++;
    return cudaGetLastError();
  }

  static const Driver* get() {
    static const Driver d = {&init,   &chunk, &bin, &materialize, &pids, &tables,
                             (int)sizeof(FEntry<P>), (int)sizeof(SEntry<P>),
                             max_blocks_model<P>(), inline_drain<P>() ? 1 : 0};
    return &d;
  }
};

}  // namespace wbrw
