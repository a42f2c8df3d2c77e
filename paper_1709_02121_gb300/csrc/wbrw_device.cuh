// wbrw_device.cuh -- device code of the signed-particle WBRW hot path for
// sm_103a (GB300), templated on the particle precision.
//
// One kernel, k_flight<P, SRC, DST>, carries the hot path of Alg. 1 (Xiong &
// Shao, arXiv:1709.02121) for a chunk of intervals [l0, L):
//   source  SRC_ARRAY  particles in the caller's SoA arrays
//           SRC_REGEN  Alg. 3 regeneration from the histogram, in registers
//           SRC_QUEUE  offspring waiting at the start of a later interval
//   flight  free streaming x <- x + (hbar/m) k dt per interval (Eq. 1) and
//           the candidate clock of constant rate gamma0 (Sec. 3.2)
//   events  candidate intervals are queued per block in shared memory and
//           processed block-cooperatively: the kick of Remark 3, the
//           acceptance (sp1) or weight (sp2/wp) cacc |sin|, the +/- pair of
//           Alg. 1 item 3 and the offspring's own events in the same interval
//   sink    DST_ARRAY  back to the arrays (offspring appended)
//           DST_BIN1   signed histogram c_nu (Eq. signed_histogram)
//           DST_BIN2   (cell, |w| in Q1.31) records for the sp2 bootstrap
//           DST_WSUM   signed weights per cell in Q1.31 (observables)
// Offspring that live into a later interval are staged in shared memory and
// appended to a queue with one global atomic per block iteration.  The next
// wave, a launch of the same kernel with SRC_QUEUE, carries them on.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "wbrw_internal.h"

namespace wbrw {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11), written from its definition.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2,
                                        uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
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
constexpr uint32_t kDrawCoins = 0xC0000000u;  // FP32 16-bit coins

// ---------------------------------------------------------------------------
// Precision traits.  FP64 arithmetic goes through the _rn intrinsics so that
// no multiply-add is contracted: every expression rounds exactly as written,
// which is the operation order the FP64 parity contract fixes.
// ---------------------------------------------------------------------------
struct P64 {
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
};

struct P32 {
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
};

template <class T>
struct FEntry {  // offspring waiting at the start of interval l
  unsigned long long pid;
  T x, k, w;
  int l;
};

template <class T>
struct EEntry {  // candidate intervals that did not fit the block's list
  unsigned long long pid;
  T x, k, w;  // x at the start of interval ls
  int ls;
  unsigned mask;  // bit b: candidate in interval l0 + b
};

static_assert(sizeof(FEntry<double>) == 40 && sizeof(FEntry<float>) == 24, "FEntry layout");
static_assert(sizeof(EEntry<double>) == 40 && sizeof(EEntry<float>) == 32, "EEntry layout");

// Kernel parameters (by value, parameter space).
template <class P>
struct KP {
  using T = typename P::T;
  T dt, dtv, hm, gamma0, cacc, sig_k, xc;
  T xmin, kmin, kmax, dx, dk, inv_dx, inv_dk;
  int nx, nk;
  double p_hi;      // FP64: u0 < p_hi may start an event in the interval
  float p_any_f;    // FP32: P(candidate) per interval
  unsigned p16;     // FP32: floor(65536 p_any)
  float p16_frac;   // FP32: 65536 p_any - p16
  uint32_t key0, key1;
  int strategy;     // 1 = sp1, 2 = sp2
  int l0, L, round;
  unsigned long long regen_base;  // epoch << 40 of the histogram's particles
  T* x;
  T* k;
  signed char* s;
  T* w;
  long long capacity;
  unsigned long long* cpid;
  FEntry<T>* fq_in;
  FEntry<T>* fq_out;
  long long qcap;
  EEntry<T>* eq;
  long long ecap;
  int* grid;
  long long* wsum;
  uint32_t* rec_cell;
  uint32_t* rec_a;
  long long rec_cap;
  const uint32_t* nz_cell;
  const unsigned long long* nz_start;
  Counters* cnt;
  wbrw_event* log;
  long long log_cap;
  int count_ledger;
};

constexpr int kItemCap = 768;   // candidate intervals per block iteration
constexpr int kStageF = 320;    // staged offspring for the next wave
constexpr int kStageOut = 192;  // staged offspring finals
constexpr int kStack = 32;      // pending offspring frames per thread
constexpr unsigned kNoItem = 0xFFFFFFFFu;

// Per-thread tallies, reduced once per block at the end of a kernel.
struct Acc {
  unsigned long long psteps, events, kill_p, kill_m, out_p, out_m;
  unsigned long long n_plus, n_minus, w_plus, w_minus;
  __device__ void zero() {
    psteps = events = kill_p = kill_m = out_p = out_m = 0;
    n_plus = n_minus = w_plus = w_minus = 0;
  }
};

template <class T>
struct Smem {
  T x[kBlock], k[kBlock], w[kBlock];
  unsigned long long pid[kBlock];
  int ls[kBlock];
  unsigned items[kItemCap];
  FEntry<T> stage_f[kStageF];
  FEntry<T> stage_out[kStageOut];
  unsigned long long win_start[kBlock + 1];
  uint32_t win_cell[kBlock + 1];
  unsigned long long red[kBlock / 32];
  unsigned long long base, total;
  int nitems, nstage_f, nstage_out;
  unsigned long long win_a;
};

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_err(Counters* c, int bit) {
  atomicOr(&c->err, bit);
}

template <class P>
__device__ __forceinline__ bool cell_of(const KP<P>& p, typename P::T x,
                                        typename P::T k, int& cell) {
  using T = typename P::T;
  const T fx = P::flr(P::mul(P::sub(x, p.xmin), p.inv_dx));
  const T fk = P::flr(P::mul(P::sub(k, p.kmin), p.inv_dk));
  if (!(fx >= (T)0 && fx < (T)p.nx && fk >= (T)0 && fk < (T)p.nk)) return false;
  cell = (int)fx * p.nk + (int)fk;
  return true;
}

// Block-wide exclusive offset of `want` items per thread into a global
// counter: one atomic per block.  Every thread of the block must call it.
template <class T>
__device__ unsigned long long block_append(Smem<T>& sm, unsigned want,
                                           unsigned long long* counter,
                                           unsigned long long& total_out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned v = want;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned t = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) sm.red[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long run = 0;
    for (int i = 0; i < kBlock / 32; ++i) {
      unsigned long long t = sm.red[i];
      sm.red[i] = run;
      run += t;
    }
    sm.base = run ? atomicAdd(counter, run) : 0ull;
    sm.total = run;
  }
  __syncthreads();
  const unsigned long long off = sm.base + sm.red[wid] + (v - want);
  total_out = sm.total;
  __syncthreads();
  return off;
}

template <class T>
__device__ void block_reduce_add(Smem<T>& sm, unsigned long long v,
                                 unsigned long long* dst) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  __syncthreads();
  if (lane == 0) sm.red[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int i = 0; i < kBlock / 32; ++i) t += sm.red[i];
    if (t) atomicAdd(dst, t);
  }
}

// ---------------------------------------------------------------------------
// Per-precision draws of the parity contract
// ---------------------------------------------------------------------------
template <class P>
struct Draw;

template <>
struct Draw<P64> {
  // Time of the first event of a segment starting at `to` (Sec. 3.2).
  __device__ static double first(const KP<P64>& p, unsigned long long pid,
                                 int l, double to, bool /*root*/) {
    const uint4 r = philox((uint32_t)pid, (uint32_t)(pid >> 32), (uint32_t)l,
                           0u, p.key0, p.key1);
    const double u0 = u53(r.x, r.y);
    return P64::add(to, P64::div(-log1p(-u0), p.gamma0));
  }
  // Event j: kick kappa ~ N(0, sig_k^2), sg = sin(2 (xe - xc) kappa),
  // acceptance uniform and the next exponential gap.
  __device__ static void event(const KP<P64>& p, unsigned long long pid,
                               int l, unsigned j, double xe, double& kap,
                               double& sg, double& u3, double& gap) {
    const uint32_t lo = (uint32_t)pid, hi = (uint32_t)(pid >> 32);
    const uint4 a = philox(lo, hi, (uint32_t)l, 1u + 2u * j, p.key0, p.key1);
    const uint4 b = philox(lo, hi, (uint32_t)l, 2u + 2u * j, p.key0, p.key1);
    const double u1 = u53(a.x, a.y), u2 = u53(a.z, a.w);
    u3 = u53(b.x, b.y);
    const double u4 = u53(b.z, b.w);
    const double z = __dmul_rn(__dsqrt_rn(__dmul_rn(-2.0, log1p(-u1))),
                               cos(__dmul_rn(6.283185307179586476925286766559, u2)));
    kap = __dmul_rn(p.sig_k, z);
    sg = sin(__dmul_rn(__dmul_rn(2.0, __dsub_rn(xe, p.xc)), kap));
    gap = __ddiv_rn(-log1p(-u4), p.gamma0);
  }
};

template <>
struct Draw<P32> {
  __device__ static float first(const KP<P32>& p, unsigned long long pid,
                                int l, float to, bool root) {
    const uint4 r = philox((uint32_t)pid, (uint32_t)(pid >> 32), (uint32_t)l,
                           0u, p.key0, p.key1);
    float u = u24(r.x);
    if (root) u *= p.p_any_f;  // the interval is known to hold an event
    return to + (-log1pf(-u)) / p.gamma0;
  }
  __device__ static void event(const KP<P32>& p, unsigned long long pid,
                               int l, unsigned j, float xe, float& kap,
                               float& sg, float& u3, float& gap) {
    const uint4 a = philox((uint32_t)pid, (uint32_t)(pid >> 32), (uint32_t)l,
                           1u + j, p.key0, p.key1);
    const float u1 = u24(a.x), u2 = u24(a.y);
    u3 = u24(a.z);
    const float u4 = u24(a.w);
    const float z = sqrtf(-2.0f * log1pf(-u1)) * cospif(2.0f * u2);
    kap = p.sig_k * z;
    sg = sinf(2.0f * (xe - p.xc) * kap);
    gap = (-log1pf(-u4)) / p.gamma0;
  }
};

// ---------------------------------------------------------------------------
// Sinks
// ---------------------------------------------------------------------------
template <class P>
__device__ __forceinline__ uint32_t q131(typename P::T w) {
  // |w| in Q1.31 (|w| <= 1): floor(|w| 2^31), exact in FP64
  return (uint32_t)floor(fabs((double)w) * 2147483648.0);
}

// A final (end-of-chunk) state produced inside the divergent event code:
// histogram sinks act directly; record / array sinks are staged.
template <class P, int DST>
__device__ void emit_child_final(const KP<P>& p, Smem<typename P::T>& sm,
                                 Acc& acc, unsigned long long pid,
                                 typename P::T x, typename P::T k,
                                 typename P::T w) {
  using T = typename P::T;
  if constexpr (DST == DST_BIN1 || DST == DST_WSUM) {
    int cell;
    if (cell_of<P>(p, x, k, cell)) {
      if constexpr (DST == DST_BIN1) atomicAdd(p.grid + cell, w > (T)0 ? 1 : -1);
      else atomicAdd((unsigned long long*)(p.wsum + cell),
                     (unsigned long long)llrint((double)w * 2147483648.0));
    } else if (p.count_ledger) {
      if (w > (T)0) ++acc.out_p; else if (w < (T)0) ++acc.out_m;
    }
    return;
  }
  const int pos = atomicAdd(&sm.nstage_out, 1);
  FEntry<T> e;
  e.pid = pid;
  e.x = x;
  e.k = k;
  e.w = w;
  e.l = p.L;
  if (pos < kStageOut) {
    sm.stage_out[pos] = e;
    return;
  }
  // rare: the stage is full, append on our own
  if constexpr (DST == DST_ARRAY) {
    const unsigned long long slot = atomicAdd(&p.cnt->n, 1ull);
    if (slot >= (unsigned long long)p.capacity) { set_err(p.cnt, ERR_CAP_PARTICLES); return; }
    p.x[slot] = x;
    p.k[slot] = k;
    p.s[slot] = w > (T)0 ? 1 : (w < (T)0 ? -1 : 0);
    if (p.w) p.w[slot] = w;
    p.cpid[slot - p.cnt->n_base] = pid;
  } else {  // DST_BIN2
    int cell;
    if (!cell_of<P>(p, x, k, cell)) {
      if (p.count_ledger) { if (w > (T)0) ++acc.out_p; else if (w < (T)0) ++acc.out_m; }
      return;
    }
    if (w == (T)0) return;
    const unsigned long long r = atomicAdd(&p.cnt->rec_len, 1ull);
    if (r >= (unsigned long long)p.rec_cap) { set_err(p.cnt, ERR_CAP_RECORDS); return; }
    const uint32_t a = q131<P>(w);
    p.rec_cell[r] = (uint32_t)cell | (w < (T)0 ? 0x80000000u : 0u);
    p.rec_a[r] = a;
    if (w > (T)0) { ++acc.n_plus; acc.w_plus += a; } else { ++acc.n_minus; acc.w_minus += a; }
  }
}

// ---------------------------------------------------------------------------
// Events of one candidate interval (Alg. 1 item 3), with every offspring's
// own events in the rest of the interval.  The root frame is the particle
// itself: its end-of-interval state belongs to the flight, not to here.
// ---------------------------------------------------------------------------
template <class T>
struct Frame {
  T xo, to, k, w;
  unsigned long long pid;
  int root;
};

template <class P, int DST>
__device__ void process_interval(const KP<P>& p, Smem<typename P::T>& sm,
                                 Acc& acc, unsigned long long pid0,
                                 typename P::T x_start, typename P::T k0,
                                 typename P::T w0, int l) {
  using T = typename P::T;
  Frame<T> stack[kStack];
  int sp = 0;
  stack[sp++] = Frame<T>{x_start, (T)0, k0, w0, pid0, 1};
  while (sp > 0) {
    const Frame<T> f = stack[--sp];
    T t = Draw<P>::first(p, f.pid, l, f.to, f.root != 0);
    unsigned j = 0;
    while (t < p.dt) {
      const T xe = P::add(f.xo, P::mul(f.k, P::mul(P::sub(t, f.to), p.hm)));
      T kap, sg, u3, gap;
      Draw<P>::event(p, f.pid, l, j, xe, kap, sg, u3, gap);
      const T fac = P::mul(p.cacc, (T)fabs(sg));
      const bool emit = p.strategy == 1 ? (u3 < fac) : (fac > (T)0);
      if (emit) {
        if (sg < (T)0) kap = -kap;
        const uint4 h = philox((uint32_t)f.pid, (uint32_t)(f.pid >> 32),
                               (uint32_t)l, kDrawPids | j, p.key0, p.key1);
        const unsigned long long pid_p =
            (1ull << 63) | ((((unsigned long long)h.y << 32) | h.x) >> 1);
        const unsigned long long pid_m =
            (1ull << 63) | ((((unsigned long long)h.w << 32) | h.z) >> 1);
        const T kp = P::add(f.k, kap), km = P::sub(f.k, kap);
        const bool kill_p = !(kp >= p.kmin && kp < p.kmax);
        const bool kill_m = !(km >= p.kmin && km < p.kmax);
        const T wc = p.strategy == 1 ? f.w : P::mul(f.w, fac);
        const T wp = wc, wm = -wc;
        ++acc.events;
        if (kill_p) { if (wp > (T)0) ++acc.kill_p; else if (wp < (T)0) ++acc.kill_m; }
        if (kill_m) { if (wm > (T)0) ++acc.kill_p; else if (wm < (T)0) ++acc.kill_m; }
        if (p.log) {
          const unsigned long long idx = atomicAdd(&p.cnt->log_len, 1ull);
          if (idx < (unsigned long long)p.log_cap) {
            wbrw_event ev;
            ev.pid = f.pid;
            ev.pid_plus = pid_p;
            ev.pid_minus = pid_m;
            ev.step = (unsigned)l;
            ev.j = j;
            ev.t = (double)t;
            ev.xe = (double)xe;
            ev.kappa = (double)kap;
            ev.factor = (double)fac;
            ev.kill_plus = kill_p;
            ev.kill_minus = kill_m;
            p.log[idx] = ev;
          }
        }
        if (!kill_p) {
          if (sp < kStack) stack[sp++] = Frame<T>{xe, t, kp, wp, pid_p, 0};
          else set_err(p.cnt, ERR_NESTING);
        }
        if (!kill_m) {
          if (sp < kStack) stack[sp++] = Frame<T>{xe, t, km, wm, pid_m, 0};
          else set_err(p.cnt, ERR_NESTING);
        }
      }
      t = P::add(t, gap);
      ++j;
    }
    if (!f.root) {
      // the offspring's position at the end of interval l
      const T xf = P::add(f.xo, P::mul(f.k, P::mul(P::sub(p.dt, f.to), p.hm)));
      if (l + 1 < p.L) {
        FEntry<T> e;
        e.pid = f.pid;
        e.x = xf;
        e.k = f.k;
        e.w = f.w;
        e.l = l + 1;
        const int pos = atomicAdd(&sm.nstage_f, 1);
        if (pos < kStageF) {
          sm.stage_f[pos] = e;
        } else {
          const unsigned long long q = atomicAdd(&p.cnt->q[p.round + 1], 1ull);
          if (q < (unsigned long long)p.qcap) p.fq_out[q] = e;
          else set_err(p.cnt, ERR_CAP_QUEUE);
        }
      } else {
        emit_child_final<P, DST>(p, sm, acc, f.pid, xf, f.k, f.w);
      }
    }
  }
}

// Flush the block's staged offspring (every thread calls).
template <class P, int DST>
__device__ void flush_stages(const KP<P>& p, Smem<typename P::T>& sm,
                             Acc& acc) {
  using T = typename P::T;
  __syncthreads();
  const int nf = min(sm.nstage_f, kStageF);
  const int no = min(sm.nstage_out, kStageOut);
  if (threadIdx.x == 0) {
    sm.base = nf ? atomicAdd(&p.cnt->q[p.round + 1], (unsigned long long)nf) : 0ull;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nf; i += kBlock) {
    const unsigned long long q = sm.base + i;
    if (q < (unsigned long long)p.qcap) p.fq_out[q] = sm.stage_f[i];
    else set_err(p.cnt, ERR_CAP_QUEUE);
  }
  __syncthreads();
  if (DST == DST_ARRAY && no > 0) {
    if (threadIdx.x == 0) sm.base = atomicAdd(&p.cnt->n, (unsigned long long)no);
    __syncthreads();
    for (int i = threadIdx.x; i < no; i += kBlock) {
      const FEntry<T> e = sm.stage_out[i];
      const unsigned long long slot = sm.base + i;
      if (slot >= (unsigned long long)p.capacity) { set_err(p.cnt, ERR_CAP_PARTICLES); continue; }
      p.x[slot] = e.x;
      p.k[slot] = e.k;
      p.s[slot] = e.w > (T)0 ? 1 : (e.w < (T)0 ? -1 : 0);
      if (p.w) p.w[slot] = e.w;
      p.cpid[slot - p.cnt->n_base] = e.pid;
    }
  } else if (DST == DST_BIN2 && no > 0) {
    // records of staged finals: compact the in-grid nonzero ones
    for (int i = threadIdx.x; i < no; i += kBlock) {
      const FEntry<T> e = sm.stage_out[i];
      int cell;
      if (!cell_of<P>(p, e.x, e.k, cell)) {
        if (p.count_ledger) { if (e.w > (T)0) ++acc.out_p; else if (e.w < (T)0) ++acc.out_m; }
        continue;
      }
      if (e.w == (T)0) continue;
      const unsigned long long r = atomicAdd(&p.cnt->rec_len, 1ull);
      if (r >= (unsigned long long)p.rec_cap) { set_err(p.cnt, ERR_CAP_RECORDS); continue; }
      const uint32_t a = q131<P>(e.w);
      p.rec_cell[r] = (uint32_t)cell | (e.w < (T)0 ? 0x80000000u : 0u);
      p.rec_a[r] = a;
      if (e.w > (T)0) { ++acc.n_plus; acc.w_plus += a; } else { ++acc.n_minus; acc.w_minus += a; }
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// The flight kernel
// ---------------------------------------------------------------------------
template <class P, int SRC, int DST>
__global__ void __launch_bounds__(kBlock) k_flight(const KP<P> p) {
  using T = typename P::T;
  __shared__ Smem<T> sm;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  Acc acc;
  acc.zero();

  unsigned long long n;
  if (SRC == SRC_ARRAY) n = p.cnt->n_src;
  else if (SRC == SRC_REGEN) n = p.cnt->regen_total;
  else n = min(p.cnt->q[p.round], (unsigned long long)p.qcap);
  const unsigned long long n_base = p.cnt->n_base, base_pid = p.cnt->base_pid;
  const unsigned long long nz = (SRC == SRC_REGEN) ? p.cnt->nz_count : 0ull;

  for (unsigned long long base = (unsigned long long)blockIdx.x * kBlock; base < n;
       base += (unsigned long long)gridDim.x * kBlock) {
    const unsigned long long slot = base + tid;
    const bool act = slot < n;
    T x = (T)0, k = (T)0, w = (T)0;
    unsigned long long pid = 0;
    int ls = p.L;

    if constexpr (SRC == SRC_REGEN) {
      // Alg. 3: slot -> its cell through the exclusive scan of |c_nu| over
      // the nonzero cells.  The block's 256 slots span at most 257 of them.
      if (tid == 0) {
        unsigned long long lo = 0, hi = nz - 1;  // last a: nz_start[a] <= base
        while (lo < hi) {
          const unsigned long long mid = lo + (hi - lo + 1) / 2;
          if (p.nz_start[mid] <= base) lo = mid; else hi = mid - 1;
        }
        sm.win_a = lo;
      }
      __syncthreads();
      const unsigned long long a0 = sm.win_a;
      for (int i = tid; i <= kBlock; i += kBlock) {
        const unsigned long long idx = a0 + i;
        sm.win_start[i] = idx < nz ? p.nz_start[idx] : ~0ull;
        sm.win_cell[i] = idx < nz ? p.nz_cell[idx] : 0u;
      }
      __syncthreads();
      if (act) {
        int lo = 0, hi = kBlock;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (sm.win_start[mid] <= slot) lo = mid; else hi = mid - 1;
        }
        const uint32_t cw = sm.win_cell[lo];
        const int cell = (int)(cw & 0x7FFFFFFFu);
        const int ix = cell / p.nk, ik = cell - ix * p.nk;
        pid = p.regen_base | slot;
        const uint4 r = philox((uint32_t)pid, (uint32_t)(pid >> 32), kStepRegen,
                               0u, p.key0, p.key1);
        T ux, uk;
        if constexpr (P::is64) { ux = (T)u53(r.x, r.y); uk = (T)u53(r.z, r.w); }
        else { ux = (T)u24(r.x); uk = (T)u24(r.y); }
        x = P::add(p.xmin, P::mul(P::add((T)ix, ux), p.dx));
        k = P::add(p.kmin, P::mul(P::add((T)ik, uk), p.dk));
        // move by single ulps back into the cell if rounding left it
        for (int it = 0; it < 8 && P::flr(P::mul(P::sub(x, p.xmin), p.inv_dx)) > (T)ix; ++it) x = P::next_dn(x);
        for (int it = 0; it < 8 && P::flr(P::mul(P::sub(x, p.xmin), p.inv_dx)) < (T)ix; ++it) x = P::next_up(x);
        for (int it = 0; it < 8 && P::flr(P::mul(P::sub(k, p.kmin), p.inv_dk)) > (T)ik; ++it) k = P::next_dn(k);
        for (int it = 0; it < 8 && P::flr(P::mul(P::sub(k, p.kmin), p.inv_dk)) < (T)ik; ++it) k = P::next_up(k);
        w = (cw >> 31) ? (T)-1 : (T)1;
        ls = p.l0;
      }
    } else if (act) {
      if constexpr (SRC == SRC_ARRAY) {
        x = p.x[slot];
        k = p.k[slot];
        w = p.w ? p.w[slot] : (T)p.s[slot];
        pid = slot < n_base ? base_pid + slot : p.cpid[slot - n_base];
        ls = p.l0;
      } else {
        const FEntry<T> e = p.fq_in[slot];
        x = e.x;
        k = e.k;
        w = e.w;
        pid = e.pid;
        ls = e.l;
      }
    }

    // ---- flight over [ls, L): streaming plus the candidate clock -------
    const T x_start = x;
    unsigned mask = 0;
    if (act) {
      const uint32_t plo = (uint32_t)pid, phi = (uint32_t)(pid >> 32);
      if constexpr (P::is64) {
        for (int l = ls; l < p.L; ++l) {
          const uint4 r = philox(plo, phi, (uint32_t)l, 0u, p.key0, p.key1);
          if (u53(r.x, r.y) < p.p_hi) mask |= 1u << (l - p.l0);
          x = P::stream(x, k, p.dtv);
        }
      } else {
        uint4 q = make_uint4(0, 0, 0, 0);
        int qb = -1;
        for (int l = ls; l < p.L; ++l) {
          const int b = l >> 3;
          if (b != qb) {
            q = philox(plo, phi, (uint32_t)b, kDrawCoins, p.key0, p.key1);
            qb = b;
          }
          const int wi = (l & 7) >> 1;
          const uint32_t word = wi == 0 ? q.x : (wi == 1 ? q.y : (wi == 2 ? q.z : q.w));
          const uint32_t coin = (l & 1) ? (word >> 16) : (word & 0xFFFFu);
          bool cand = coin < p.p16;
          if (coin == p.p16) {
            const uint4 r = philox(plo, phi, (uint32_t)l, 0u, p.key0, p.key1);
            cand = u24(r.y) < p.p16_frac;
          }
          if (cand) mask |= 1u << (l - p.l0);
          x = P::stream(x, k, p.dtv);
        }
      }
      acc.psteps += (unsigned long long)(p.L - ls);
    }

    if (tid == 0) {
      sm.nitems = 0;
      sm.nstage_f = 0;
      sm.nstage_out = 0;
    }
    sm.x[tid] = x_start;
    sm.k[tid] = k;
    sm.w[tid] = w;
    sm.pid[tid] = pid;
    sm.ls[tid] = ls;

    // ---- the particle's own final state --------------------------------
    if constexpr (DST == DST_ARRAY) {
      if constexpr (SRC == SRC_ARRAY) {
        if (act) p.x[slot] = x;
        __syncthreads();
      } else if constexpr (SRC == SRC_REGEN) {
        if (act && slot >= (unsigned long long)p.capacity) {
          set_err(p.cnt, ERR_CAP_PARTICLES);
        } else if (act) {
          p.x[slot] = x;
          p.k[slot] = k;
          p.s[slot] = w > (T)0 ? 1 : -1;
          if (p.w) p.w[slot] = w;
        }
        __syncthreads();
      } else {
        unsigned long long tot;
        const unsigned long long off = block_append<T>(sm, act ? 1u : 0u, &p.cnt->n, tot);
        if (act) {
          if (off >= (unsigned long long)p.capacity) {
            set_err(p.cnt, ERR_CAP_PARTICLES);
          } else {
            p.x[off] = x;
            p.k[off] = k;
            p.s[off] = w > (T)0 ? 1 : (w < (T)0 ? -1 : 0);
            if (p.w) p.w[off] = w;
            p.cpid[off - n_base] = pid;
          }
        }
      }
    } else if constexpr (DST == DST_BIN1) {
      long long key = -1;
      if (act) {
        int cell;
        if (cell_of<P>(p, x, k, cell)) key = 2ll * cell + (w > (T)0 ? 1 : 0);
        else if (p.count_ledger) { if (w > (T)0) ++acc.out_p; else ++acc.out_m; }
      }
      const unsigned grp = __match_any_sync(0xFFFFFFFFu, (unsigned long long)key);
      if (key >= 0 && lane == __ffs(grp) - 1)
        atomicAdd(p.grid + (key >> 1), (key & 1) ? __popc(grp) : -__popc(grp));
      __syncthreads();
    } else if constexpr (DST == DST_WSUM) {
      if (act) {
        int cell;
        if (cell_of<P>(p, x, k, cell))
          atomicAdd((unsigned long long*)(p.wsum + cell),
                    (unsigned long long)llrint((double)w * 2147483648.0));
      }
      __syncthreads();
    } else {  // DST_BIN2
      int cell = -1;
      if (act) {
        if (!cell_of<P>(p, x, k, cell)) {
          cell = -1;
          if (p.count_ledger) { if (w > (T)0) ++acc.out_p; else if (w < (T)0) ++acc.out_m; }
        } else if (w == (T)0) {
          cell = -1;
        }
      }
      unsigned long long tot;
      const unsigned long long r = block_append<T>(sm, cell >= 0 ? 1u : 0u, &p.cnt->rec_len, tot);
      if (cell >= 0) {
        if (r >= (unsigned long long)p.rec_cap) {
          set_err(p.cnt, ERR_CAP_RECORDS);
        } else {
          const uint32_t a = q131<P>(w);
          p.rec_cell[r] = (uint32_t)cell | (w < (T)0 ? 0x80000000u : 0u);
          p.rec_a[r] = a;
          if (w > (T)0) { ++acc.n_plus; acc.w_plus += a; } else { ++acc.n_minus; acc.w_minus += a; }
        }
      }
    }

    // ---- candidate intervals -> the block's list (or the overflow queue)
    const int cnt = __popc(mask);
    if (cnt) {
      const int pos = atomicAdd(&sm.nitems, cnt);
      if (pos + cnt <= kItemCap) {
        unsigned m = mask;
        for (int i = 0; i < cnt; ++i) {
          const int b = __ffs(m) - 1;
          m &= m - 1;
          sm.items[pos + i] = (unsigned)tid | ((unsigned)b << 16);
        }
      } else {
        for (int i = pos; i < kItemCap; ++i) sm.items[i] = kNoItem;
        const unsigned long long e = atomicAdd(&p.cnt->e[p.round], 1ull);
        if (e < (unsigned long long)p.ecap) {
          EEntry<T> ee;
          ee.pid = pid;
          ee.x = x_start;
          ee.k = k;
          ee.w = w;
          ee.ls = ls;
          ee.mask = mask;
          p.eq[e] = ee;
        } else {
          set_err(p.cnt, ERR_CAP_EQUEUE);
        }
      }
    }
    __syncthreads();

    // ---- process them, one per thread ----------------------------------
    const int ni = min(sm.nitems, kItemCap);
    for (int i = tid; i < ni; i += kBlock) {
      const unsigned it = sm.items[i];
      if (it == kNoItem) continue;
      const int owner = (int)(it & 0xFFFFu);
      const int l = p.l0 + (int)(it >> 16);
      const T ko = sm.k[owner];
      T xs = sm.x[owner];
      for (int ll = sm.ls[owner]; ll < l; ++ll) xs = P::stream(xs, ko, p.dtv);
      process_interval<P, DST>(p, sm, acc, sm.pid[owner], xs, ko, sm.w[owner], l);
    }
    flush_stages<P, DST>(p, sm, acc);
  }

  // ---- tallies ------------------------------------------------------------
  block_reduce_add<T>(sm, acc.psteps, &p.cnt->ledger[SRC == SRC_QUEUE ? LG_PSTEPS : LG_PSTEPS0]);
  block_reduce_add<T>(sm, acc.events, &p.cnt->ledger[LG_EVENTS]);
  block_reduce_add<T>(sm, acc.kill_p, &p.cnt->ledger[LG_KILL_P]);
  block_reduce_add<T>(sm, acc.kill_m, &p.cnt->ledger[LG_KILL_M]);
  block_reduce_add<T>(sm, acc.out_p, &p.cnt->ledger[LG_OUT_P]);
  block_reduce_add<T>(sm, acc.out_m, &p.cnt->ledger[LG_OUT_M]);
  if constexpr (DST == DST_BIN2) {
    block_reduce_add<T>(sm, acc.n_plus, &p.cnt->boot_n[0]);
    block_reduce_add<T>(sm, acc.n_minus, &p.cnt->boot_n[1]);
    block_reduce_add<T>(sm, acc.w_plus, &p.cnt->boot_w[0]);
    block_reduce_add<T>(sm, acc.w_minus, &p.cnt->boot_w[1]);
  }
}

// Candidate intervals that overflowed a block's list in round `p.round`.
template <class P, int DST>
__global__ void __launch_bounds__(kBlock) k_event(const KP<P> p) {
  using T = typename P::T;
  __shared__ Smem<T> sm;
  Acc acc;
  acc.zero();
  const unsigned long long n = min(p.cnt->e[p.round], (unsigned long long)p.ecap);
  for (unsigned long long base = (unsigned long long)blockIdx.x * kBlock; base < n;
       base += (unsigned long long)gridDim.x * kBlock) {
    if (threadIdx.x == 0) {
      sm.nstage_f = 0;
      sm.nstage_out = 0;
    }
    __syncthreads();
    const unsigned long long i = base + threadIdx.x;
    if (i < n) {
      const EEntry<T> e = p.eq[i];
      unsigned m = e.mask;
      T xs = e.x;
      int ll = e.ls;
      while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        const int l = p.l0 + b;
        for (; ll < l; ++ll) xs = P::stream(xs, e.k, p.dtv);
        process_interval<P, DST>(p, sm, acc, e.pid, xs, e.k, e.w, l);
      }
    }
    flush_stages<P, DST>(p, sm, acc);
  }
  block_reduce_add<T>(sm, acc.events, &p.cnt->ledger[LG_EVENTS]);
  block_reduce_add<T>(sm, acc.kill_p, &p.cnt->ledger[LG_KILL_P]);
  block_reduce_add<T>(sm, acc.kill_m, &p.cnt->ledger[LG_KILL_M]);
  block_reduce_add<T>(sm, acc.out_p, &p.cnt->ledger[LG_OUT_P]);
  block_reduce_add<T>(sm, acc.out_m, &p.cnt->ledger[LG_OUT_M]);
  if constexpr (DST == DST_BIN2) {
    block_reduce_add<T>(sm, acc.n_plus, &p.cnt->boot_n[0]);
    block_reduce_add<T>(sm, acc.n_minus, &p.cnt->boot_n[1]);
    block_reduce_add<T>(sm, acc.w_plus, &p.cnt->boot_w[0]);
    block_reduce_add<T>(sm, acc.w_minus, &p.cnt->boot_w[1]);
  }
}

// Initial particles from the Gaussian-wavepacket Wigner function (positive):
// Box-Muller on the init stream of pid = slot, x ~ N(x0, sx^2), k ~ N(k0, sk^2).
template <class P>
__global__ void __launch_bounds__(kBlock) k_init(const KP<P> p,
                                                 unsigned long long n,
                                                 double x0, double sx,
                                                 double k0, double sk) {
  using T = typename P::T;
  for (unsigned long long i = (unsigned long long)blockIdx.x * kBlock + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * kBlock) {
    const uint4 r = philox((uint32_t)i, (uint32_t)(i >> 32), kStepInit, 0u,
                           p.key0, p.key1);
    T x, k;
    if constexpr (P::is64) {
      const double ua = u53(r.x, r.y), ub = u53(r.z, r.w);
      const double rad = __dsqrt_rn(__dmul_rn(-2.0, log1p(-ua)));
      const double th = __dmul_rn(6.283185307179586476925286766559, ub);
      x = (T)__dadd_rn(x0, __dmul_rn(sx, __dmul_rn(rad, cos(th))));
      k = (T)__dadd_rn(k0, __dmul_rn(sk, __dmul_rn(rad, sin(th))));
    } else {
      const float ua = u24(r.x), ub = u24(r.y);
      const float rad = sqrtf(-2.0f * log1pf(-ua));
      float sn, cs;
      sincospif(2.0f * ub, &sn, &cs);
      x = (T)(x0 + sx * (double)(rad * cs));
      k = (T)(k0 + sk * (double)(rad * sn));
    }
    p.x[i] = x;
    p.k[i] = k;
    p.s[i] = 1;
    if (p.w) p.w[i] = (T)1;
  }
}

// Stream ids of the materialised particles.
template <class P>
__global__ void __launch_bounds__(kBlock) k_pids(const KP<P> p,
                                                 unsigned long long* out) {
  const unsigned long long n = p.cnt->n, nb = p.cnt->n_base, bp = p.cnt->base_pid;
  for (unsigned long long i = (unsigned long long)blockIdx.x * kBlock + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * kBlock)
    out[i] = i < nb ? bp + i : p.cpid[i - nb];
}

}  // namespace wbrw

// ---------------------------------------------------------------------------
// Host-side driver of the kernels above for one precision.
// ---------------------------------------------------------------------------
namespace wbrw {

template <class P>
KP<P> make_kp(const Ctx* c) {
  using T = typename P::T;
  KP<P> p;
  const wbrw_config& g = c->cfg;
  p.dt = (T)g.dt;
  p.dtv = (T)c->dtv;
  p.hm = (T)c->hm;
  p.gamma0 = (T)c->gamma0;
  p.cacc = (T)c->cacc;
  p.sig_k = (T)c->sig_k;
  p.xc = (T)c->pot.xc;
  p.xmin = (T)g.xmin;
  p.kmin = (T)g.kmin;
  p.kmax = (T)g.kmax;
  p.dx = (T)c->dx;
  p.dk = (T)c->dk;
  p.inv_dx = (T)c->inv_dx;
  p.inv_dk = (T)c->inv_dk;
  p.nx = g.nx;
  p.nk = g.nk;
  p.p_hi = c->p_any * (1.0 + 1e-9) + 1e-300;
  p.p_any_f = (float)c->p_any;
  const double sc = c->p_any * 65536.0;
  const double fl = floor(sc);
  p.p16 = (unsigned)fl;
  p.p16_frac = (float)(sc - fl);
  p.key0 = (uint32_t)g.seed;
  p.key1 = (uint32_t)(g.seed >> 32);
  p.strategy = g.strategy;
  p.l0 = p.L = (int)c->step;
  p.round = 0;
  p.regen_base = (unsigned long long)c->epoch << 40;
  p.x = (T*)c->buf.x;
  p.k = (T*)c->buf.k;
  p.s = c->buf.s;
  p.w = g.strategy == WBRW_SP2_BOOTSTRAP ? (T*)c->buf.w : nullptr;
  p.capacity = c->buf.capacity;
  p.cpid = c->cpid;
  p.fq_in = (FEntry<T>*)c->fq[0];
  p.fq_out = (FEntry<T>*)c->fq[1];
  p.qcap = c->qcap;
  p.eq = (EEntry<T>*)c->eq;
  p.ecap = c->ecap;
  p.grid = c->buf.grid;
  p.wsum = c->tmp_wsum;
  p.rec_cell = c->rec_cell;
  p.rec_a = c->rec_a;
  p.rec_cap = c->rec_cap;
  p.nz_cell = c->nz_cell;
  p.nz_start = c->nz_start;
  p.cnt = c->cnt;
  p.log = (wbrw_event*)c->buf.event_log;
  p.log_cap = c->buf.event_log ? c->buf.event_log_capacity : 0;
  p.count_ledger = 1;
  return p;
}

template <class K>
int grid_for(Ctx* c, K kern) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * c->num_sms;
}

template <class P, int SRC, int DST>
cudaError_t flight(Ctx* c, const KP<P>& p) {
  static int grid = 0;
  if (!grid) grid = grid_for(c, k_flight<P, SRC, DST>);
  k_flight<P, SRC, DST><<<grid, kBlock, 0, c->stream>>>(p);
  c->launches++;
  return cudaGetLastError();
}

template <class P, int DST>
cudaError_t events(Ctx* c, const KP<P>& p) {
  static int grid = 0;
  if (!grid) grid = grid_for(c, k_event<P, DST>);
  k_event<P, DST><<<grid, kBlock, 0, c->stream>>>(p);
  c->launches++;
  return cudaGetLastError();
}

template <class P, int DST>
cudaError_t flight_src(Ctx* c, const KP<P>& p, int src) {
  switch (src) {
    case SRC_ARRAY: return flight<P, SRC_ARRAY, DST>(c, p);
    case SRC_REGEN: return flight<P, SRC_REGEN, DST>(c, p);
    default: return flight<P, SRC_QUEUE, DST>(c, p);
  }
}

template <class P>
cudaError_t flight_any(Ctx* c, const KP<P>& p, int src, int dst) {
  switch (dst) {
    case DST_ARRAY: return flight_src<P, DST_ARRAY>(c, p, src);
    case DST_BIN1: return flight_src<P, DST_BIN1>(c, p, src);
    case DST_BIN2: return flight_src<P, DST_BIN2>(c, p, src);
    default: return flight_src<P, DST_WSUM>(c, p, src);
  }
}

template <class P>
cudaError_t events_any(Ctx* c, const KP<P>& p, int dst) {
  switch (dst) {
    case DST_ARRAY: return events<P, DST_ARRAY>(c, p);
    case DST_BIN1: return events<P, DST_BIN1>(c, p);
    case DST_BIN2: return events<P, DST_BIN2>(c, p);
    default: return events<P, DST_WSUM>(c, p);
  }
}

template <class P>
struct DriverImpl {
  static cudaError_t init(Ctx* c, long long n, double x0, double sx, double k0) {
    cudaError_t e = launch_setup(c, SETUP_INIT, (unsigned long long)n, 0);
    if (e != cudaSuccess) return e;
    KP<P> p = make_kp<P>(c);
    static int grid = 0;
    if (!grid) grid = grid_for(c, k_init<P>);
    const double sk = 1.0 / (2.0 * sx);
    k_init<P><<<grid, kBlock, 0, c->stream>>>(p, (unsigned long long)n, x0, sx, k0, sk);
    c->launches++;
    return cudaGetLastError();
  }

  // Intervals [l0, L): round r carries the particles that start at l0 + r
  // or later; offspring start one interval after their birth, so L - l0
  // rounds drain every wave.
  static cudaError_t chunk(Ctx* c, int l0, int L, int src, int dst) {
    cudaError_t e = launch_setup(c, SETUP_CHUNK, 0, 0);
    if (e != cudaSuccess) return e;
    KP<P> p = make_kp<P>(c);
    p.l0 = l0;
    p.L = L;
    const int rounds = L > l0 ? L - l0 : 1;
    for (int r = 0; r < rounds; ++r) {
      p.round = r;
      p.fq_in = (FEntry<typename P::T>*)c->fq[r & 1];
      p.fq_out = (FEntry<typename P::T>*)c->fq[(r + 1) & 1];
      if (r == 0) prof_begin(c);
      e = flight_any<P>(c, p, r == 0 ? src : (int)SRC_QUEUE, dst);
      if (r == 0) prof_end(c);
      if (e != cudaSuccess) return e;
      if (L > l0) {
        e = events_any<P>(c, p, dst);
        if (e != cudaSuccess) return e;
      }
    }
    return cudaSuccess;
  }

  static cudaError_t bin(Ctx* c, int dst, int* grid, int count_ledger) {
    cudaError_t e = launch_setup(c, SETUP_CHUNK, 0, 0);
    if (e != cudaSuccess) return e;
    KP<P> p = make_kp<P>(c);
    p.grid = grid;
    p.count_ledger = count_ledger;
    return flight_any<P>(c, p, SRC_ARRAY, dst);
  }

  static cudaError_t materialize(Ctx* c) {
    cudaError_t e = launch_setup(c, SETUP_AFTER_REGEN,
                                 (unsigned long long)c->epoch << 40, 0);
    if (e != cudaSuccess) return e;
    KP<P> p = make_kp<P>(c);
    return flight<P, SRC_REGEN, DST_ARRAY>(c, p);
  }

  static cudaError_t pids(Ctx* c, unsigned long long* out) {
    KP<P> p = make_kp<P>(c);
    static int grid = 0;
    if (!grid) grid = grid_for(c, k_pids<P>);
    k_pids<P><<<grid, kBlock, 0, c->stream>>>(p, out);
    c->launches++;
    return cudaGetLastError();
  }

  static const Driver* get() {
    static const Driver d = {&init, &chunk, &bin, &materialize, &pids};
    return &d;
  }
};

}  // namespace wbrw
