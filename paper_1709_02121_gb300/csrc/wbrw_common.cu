// wbrw_common.cu -- precision-independent kernels of the resampling step:
// the cell scans that turn a signed histogram into the regeneration plan of
// Alg. 3, the signed residual bootstrap of sp2 (Alg. 2 with Eq. lambda and
// Eq. double_bootstrap / boostrap_histogram) and the observables of
// Eq. estimator.  All counts are integers and all sums that decide a count
// are in fixed point, so the results do not depend on thread order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "wbrw_internal.h"

namespace wbrw {

namespace {

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

constexpr uint32_t kStepBoot = 0xFFFFFFFDu;
constexpr uint32_t kStepRound = 0xFFFFFFFCu;

// ---------------------------------------------------------------------------
// Counter set-up (one thread).
// ---------------------------------------------------------------------------
__global__ void k_setup(Counters* c, int op, unsigned long long a,
                        unsigned long long b) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  switch (op) {
    case SETUP_CHUNK:
      c->n_src = c->n;
      c->per_l0 = (int)a;
      c->per_regen_base = b;
      break;
    case SETUP_CHUNK_DEV:
      c->n_src = c->n;
      break;
    case SETUP_PERIOD:
      c->per_l0 = (int)a;
      c->per_regen_base = b;
      break;
    case SETUP_ADVANCE:
      c->per_l0 += (int)a;
      c->per_regen_base += 1ull << 40;
      break;
    case SETUP_AFTER_REGEN:
      c->n = c->regen_total;
      c->n_base = c->regen_total;
      c->base_pid = a;
      c->per_regen_base = a;
      c->per_l0 = (int)b;
      break;
    case SETUP_INIT:
      c->n = a;
      c->n_base = a;
      c->base_pid = 0;
      break;
    case SETUP_BOOT:
      for (int s = 0; s < 2; ++s) {
        c->boot_n[s] = c->boot_w[s] = c->boot_keep[s] = c->boot_nr[s] = 0;
        c->boot_R[s] = 0;
      }
      break;
  }
}

// ---------------------------------------------------------------------------
// Block-wide exclusive scan of one u64 per thread (kBlock threads).
// ---------------------------------------------------------------------------
__device__ unsigned long long block_exscan(unsigned long long v,
                                           unsigned long long* red,
                                           unsigned long long& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) red[wid] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long run = 0;
    for (int i = 0; i < kBlock / 32; ++i) {
      const unsigned long long t = red[i];
      red[i] = run;
      run += t;
    }
    red[kBlock / 32] = run;
  }
  __syncthreads();
  const unsigned long long ex = red[wid] + inc - v;
  total = red[kBlock / 32];
  __syncthreads();
  return ex;
}

// ---------------------------------------------------------------------------
// Histogram -> regeneration plan (Alg. 3 without rounding): n_nu = |c_nu|,
// exclusive scan over cells, compact list of the nonzero cells with their
// first slot.  Three passes over tiles of kScanTile cells.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_cells_a(const int* grid, long long nh,
                                                    unsigned long long* bsum,
                                                    unsigned int* bnz) {
  __shared__ unsigned long long red[kBlock / 32 + 1];
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  unsigned long long s = 0, z = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const long long c = base + i;
    if (c < nh) {
      const int v = grid[c];
      s += (unsigned long long)(v < 0 ? -(long long)v : (long long)v);
      z += v != 0;
    }
  }
  unsigned long long ts, tz;
  block_exscan(s, red, ts);
  block_exscan(z, red, tz);
  if (threadIdx.x == 0) {
    bsum[blockIdx.x] = ts;
    bnz[blockIdx.x] = (unsigned int)tz;
  }
}

// which = 0: the plan of the signed particles; 1: the tangent plan.
__global__ void __launch_bounds__(kBlock) k_cells_b(unsigned long long* bsum,
                                                    unsigned int* bnz,
                                                    long long nb, Counters* c,
                                                    long long tile_cap,
                                                    unsigned long long* inst_end, int which) {
  __shared__ unsigned long long red[kBlock / 32 + 1];
  unsigned long long carry_s = 0, carry_z = 0;
  for (long long b0 = 0; b0 < nb; b0 += kBlock) {
    const long long b = b0 + threadIdx.x;
    const unsigned long long s = b < nb ? bsum[b] : 0, z = b < nb ? bnz[b] : 0;
    unsigned long long ts, tz;
    const unsigned long long es = block_exscan(s, red, ts);
    const unsigned long long ez = block_exscan(z, red, tz);
    if (b < nb) {
      bsum[b] = carry_s + es;
      bnz[b] = (unsigned int)(carry_z + ez);
    }
    carry_s += ts;
    carry_z += tz;
  }
  if (threadIdx.x == 0) {
    if (which) {
      c->tan_total = carry_s;
      c->tan_nz = carry_z;
    } else {
      c->regen_total = carry_s;
      c->nz_count = carry_z;
    }
    *inst_end = carry_s;
    if (carry_s > (unsigned long long)tile_cap * 32ull) atomicOr(&c->err, ERR_CAP_PARTICLES);
  }
}

// Also records the first slot of each instance (cells i nhi .. (i+1) nhi - 1
// belong to instance i) in inst_slot.
__global__ void __launch_bounds__(kBlock) k_cells_c(const int* grid, long long nh,
                                                    const unsigned long long* bsum,
                                                    const unsigned int* bnz,
                                                    uint32_t* nz_cell,
                                                    unsigned long long* nz_start,
                                                    uint32_t* tile_nz, long long tile_cap,
                                                    long long nhi,
                                                    unsigned long long* inst_slot) {
  __shared__ unsigned long long red[kBlock / 32 + 1];
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  int v[kScanItems];
  unsigned long long s = 0, z = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const long long c = base + i;
    v[i] = c < nh ? grid[c] : 0;
    s += (unsigned long long)(v[i] < 0 ? -(long long)v[i] : (long long)v[i]);
    z += v[i] != 0;
  }
  unsigned long long ts, tz;
  unsigned long long os = block_exscan(s, red, ts) + bsum[blockIdx.x];
  unsigned long long oz = block_exscan(z, red, tz) + bnz[blockIdx.x];
  long long next_inst = (base + nhi - 1) / nhi * nhi;  // first instance boundary >= base
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i == next_inst && next_inst < nh) {
      inst_slot[next_inst / nhi] = os;
      next_inst += nhi;
    }
    // every 32-slot tile whose first slot falls in this cell starts here:
    // tiles [t0, t1) (tile indices fit 32 bits: tile_cap <= capacity / 32 + 2)
    unsigned t0 = 0, t1 = 0;
    const uint32_t val = (uint32_t)oz;
    if (v[i] != 0) {
      const unsigned long long m = (unsigned long long)(v[i] < 0 ? -(long long)v[i] : (long long)v[i]);
      nz_cell[oz] = (uint32_t)(base + i) | (v[i] < 0 ? 0x80000000u : 0u);
      nz_start[oz] = os;
      t0 = (unsigned)min((os + 31) >> 5, (unsigned long long)tile_cap);
      t1 = (unsigned)min((os + m + 31) >> 5, (unsigned long long)tile_cap);
      ++oz;
      os += m;
    }
    // the warp writes each lane's tile range in turn, 32 consecutive
    // entries per store (a dense cell spans many tiles)
    for (unsigned pend = __ballot_sync(0xFFFFFFFFu, t1 > t0); pend; pend &= pend - 1) {
      const int src = __ffs(pend) - 1;
      const unsigned a = __shfl_sync(0xFFFFFFFFu, t0, src), b = __shfl_sync(0xFFFFFFFFu, t1, src);
      const uint32_t w = __shfl_sync(0xFFFFFFFFu, val, src);
      for (unsigned t = a + lane; t < b; t += 32) tile_nz[t] = w;
    }
  }
}

// ---------------------------------------------------------------------------
// In-place inclusive scan of a u64 array (per-cell bootstrap residuals).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_u64_a(const unsigned long long* a, long long n,
                                                  unsigned long long* bsum) {
  __shared__ unsigned long long red[kBlock / 32 + 1];
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  unsigned long long s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) s += a[base + i];
  unsigned long long t;
  block_exscan(s, red, t);
  if (threadIdx.x == 0) bsum[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kBlock) k_u64_b(unsigned long long* bsum, long long nb,
                                                  unsigned long long* total) {
  __shared__ unsigned long long red[kBlock / 32 + 1];
  unsigned long long carry = 0;
  for (long long b0 = 0; b0 < nb; b0 += kBlock) {
    const long long b = b0 + threadIdx.x;
    const unsigned long long s = b < nb ? bsum[b] : 0;
    unsigned long long t;
    const unsigned long long e = block_exscan(s, red, t);
    if (b < nb) bsum[b] = carry + e;
    carry += t;
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kBlock) k_u64_c(unsigned long long* a, long long n,
                                                  const unsigned long long* bsum) {
  __shared__ unsigned long long red[kBlock / 32 + 1];
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  unsigned long long v[kScanItems];
  unsigned long long s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < n ? a[base + i] : 0;
    s += v[i];
  }
  unsigned long long t;
  unsigned long long run = block_exscan(s, red, t) + bsum[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    run += v[i];
    if (base + i < n) a[base + i] = run;
  }
}

// ---------------------------------------------------------------------------
// sp2 bootstrap (Alg. 2 per side).  Records hold (cell | side << 31, a) with
// a = floor(|w| 2^31); N^s and W^s = sum a were tallied with the records.
// ---------------------------------------------------------------------------
constexpr int kBootChunk = 1024;  // records per work item of k_boot_bin
constexpr int kBootBinBlocks = 8; // resident blocks per SM k_boot_bin is built and launched for
constexpr int kBootBinBatchBlocks = 6;  // the same for its batch form (shares from a table)
constexpr int kTallyLoads = 4;          // groups of 32 records k_bootb_tally loads ahead
constexpr int kTallyBlocks = 5;         // resident blocks per SM of k_bootb_tally (bound and grid)

// The share q_i = a_i N^s / W^s of a record of side s (Alg. 2 on S^s), split
// into its integer part and its Q0.32 residual.  fx (FP32 runs): in fixed
// point, a_i M / 2^64 with M = floor(N 2^64 / W) from one FP64 division, so
// that no record needs FP64 arithmetic (slow on this GPU); the integer part
// and the residual agree with the FP64 form to about one unit of 2^-32 (the
// FP32 contract is in law).  FP64 runs keep the FP64 form, which the oracle
// follows.  The two sides' constants are separate scalars, chosen by a
// select: an array indexed by the side would live in local memory.
struct BootShare {
  double ratio0, ratio1;
  unsigned long long mx0, mx1;
  bool fx0, fx1;

  __device__ void init(const Counters* c, int fx) { init(c->boot_n, c->boot_w, fx); }
  // from the counts N^s and the weight sums W^s (Q1.31) of the two sides
  __device__ void init(const unsigned long long* bn, const unsigned long long* bw, int fx) {
    ratio0 = ratio1 = 0.0;
    mx0 = mx1 = 0;
    fx0 = fx1 = false;
    for (int s = 0; s < 2; ++s) {
      const double r = bw[s] > 0 ? __ddiv_rn((double)bn[s], (double)bw[s]) : 0.0;
      unsigned long long m_s = 0;
      bool f_s = false;
      if (fx && bn[s] < bw[s]) {
        const double m = r * 18446744073709551616.0;
        if (m < 18446744073709551616.0) {
          m_s = (unsigned long long)m;
          f_s = true;
        }
      }
      if (s == 0) { ratio0 = r; mx0 = m_s; fx0 = f_s; } else { ratio1 = r; mx1 = m_s; fx1 = f_s; }
    }
  }
  __device__ __forceinline__ void of(uint32_t a, int side, int& kf,
                                     unsigned long long& res) const {
    if (side ? fx1 : fx0) {
      const unsigned long long m = side ? mx1 : mx0;
      kf = (int)__umul64hi((unsigned long long)a, m);  // bits 64..95 of the 96-bit a m
      res = ((unsigned long long)a * m) >> 32;         // bits 32..63: the Q0.32 residual
    } else {
      const double q = __dmul_rn((double)a, side ? ratio1 : ratio0);
      const double fl = floor(q);
      res = (unsigned long long)floor(__dmul_rn(__dsub_rn(q, fl), 4294967296.0));
      kf = (int)fl;
    }
  }
};

// An instance's shares (its record filled by k_bootb_share).
__device__ __forceinline__ BootShare share_of(const BootInst& b) {
  BootShare sh;
  sh.ratio0 = b.ratio[0];
  sh.ratio1 = b.ratio[1];
  sh.mx0 = b.mx[0];
  sh.mx1 = b.mx[1];
  sh.fx0 = b.fx[0] != 0;
  sh.fx1 = b.fx[1] != 0;
  return sh;
}

// The regenerated particles' part (weight +-1, a = 2^31, all of a side with
// the same share): count x (integer part, residual) per side and cell,
// written into the tallies that k_boot_bin then adds the records to.
__global__ void __launch_bounds__(kBlock) k_boot_unit(Counters* c, const int* ucnt, long long nh,
                                                      int* keep0, int* keep1,
                                                      unsigned long long* res0,
                                                      unsigned long long* res1, int fx) {
  __shared__ unsigned long long red[kBlock / 32 + 1];
  BootShare sh;
  sh.init(c, fx);
  int kf[2];
  unsigned long long rs[2];
  sh.of(2147483648u, 0, kf[0], rs[0]);
  sh.of(2147483648u, 1, kf[1], rs[1]);
  unsigned long long ks0 = 0, ks1 = 0;
  for (long long nu = (long long)blockIdx.x * kBlock + threadIdx.x; nu < nh;
       nu += (long long)gridDim.x * kBlock) {
    const int u0 = ucnt[nu], u1 = ucnt[nh + nu];
    keep0[nu] = u0 * kf[0];
    keep1[nu] = u1 * kf[1];
    res0[nu] = (unsigned long long)u0 * rs[0];
    res1[nu] = (unsigned long long)u1 * rs[1];
    ks0 += (unsigned long long)u0 * (unsigned long long)kf[0];
    ks1 += (unsigned long long)u1 * (unsigned long long)kf[1];
  }
  for (int s = 0; s < 2; ++s) {
    unsigned long long t;
    block_exscan(s ? ks1 : ks0, red, t);
    if (threadIdx.x == 0 && t) atomicAdd(&c->boot_keep[s], t);
  }
}

// The instance of global cell nu (< 2^30) when every instance owns nhi
// cells: floor(nu / nhi) from one multiply by mag = ceil(2^40 / nhi) (whose
// estimate exceeds the quotient by at most one, since nu (mag - 2^40 / nhi)
// < 2^-10 2^40) and one correction, instead of an integer division.
__device__ __forceinline__ unsigned long long inst_magic(int nhi) {
  return ((1ull << 40) + (unsigned long long)nhi - 1ull) / (unsigned long long)nhi;
}
__device__ __forceinline__ unsigned inst_of_cell(unsigned nu, int nhi, unsigned long long mag) {
  unsigned q = (unsigned)(((unsigned long long)nu * mag) >> 40);
  if (q * (unsigned)nhi > nu) --q;
  return q;
}

// The offspring records' shares added to the cell tallies.  BATCH: the
// records of all instances of a batch, each with its instance's share (the
// instance of global cell nu is nu / nhi); the instances' sums of the
// integer parts are then taken over their cells (k_bootb_keep), not here.
template <bool BATCH>
__global__ void __launch_bounds__(kBlock, BATCH ? kBootBinBatchBlocks : kBootBinBlocks)
    k_boot_bin(Counters* c, const uint32_t* rec_cell, const uint32_t* rec_a, const unsigned* rcnt,
               int nseg, long long rseg, int* keep0, int* keep1, unsigned long long* res0,
               unsigned long long* res1, int fx, BootInst* bi, int ninst, int nhi) {
  const unsigned long long mag = inst_magic(nhi);
  __shared__ unsigned long long red[kBlock / 32 + 1];
  __shared__ BootShare tab[BATCH ? kMaxInst : 1];
  BootShare sh;
  if constexpr (BATCH) {
    for (int i = threadIdx.x; i < ninst; i += kBlock) tab[i] = share_of(bi[i]);
    __syncthreads();
  } else {
    sh.init(c, fx);
  }
  unsigned long long ks0 = 0, ks1 = 0;
  // records sit in one segment per producer warp; a warp takes a segment
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * kBlock + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * kBlock) >> 5;
  // Records of one producer segment are mostly in cell order (the first
  // wave writes a regenerated tile's particles in order), so the warp sums
  // runs of equal (cell, side) keys in consecutive lanes and only a run's
  // first lane adds to the grids: far fewer contended atomics, the same
  // integer sums.
  // Work items: chunks of kBootChunk records of a segment, spread over all
  // warps (a segment holds up to rseg records; most chunks of the last
  // segments are empty)
  const long long cps = (rseg + kBootChunk - 1) / kBootChunk;
  for (long long it = gw; it < (long long)nseg * cps; it += nw) {
    const long long sg = it / cps;
    const unsigned b0 = (unsigned)((it - sg * cps) * kBootChunk);
    const unsigned n = min(min(rcnt[sg], (unsigned)rseg), b0 + (unsigned)kBootChunk);
    const uint32_t* rcs = rec_cell + sg * rseg;  // the segment's records
    const uint32_t* ras = rec_a + sg * rseg;
    // the batch form loads kBinLoads groups of 32 records before it uses the
    // first (its atomics scatter over arrays larger than L2, and it waits on
    // the record loads otherwise)
    constexpr int kBinLoads = BATCH ? 4 : 1;
    for (unsigned b = b0; b < n; b += 32u * kBinLoads) {
     uint32_t rcv[kBinLoads], rav[kBinLoads];
#pragma unroll
     for (int j = 0; j < kBinLoads; ++j) {
       const unsigned i = b + 32u * j + lane;
       if constexpr (BATCH) {
         rcv[j] = i < n ? __ldcs(rcs + i) : ~0u;
         rav[j] = i < n ? __ldcs(ras + i) : 0u;
       } else {
         rcv[j] = i < n ? rcs[i] : ~0u;
         rav[j] = i < n ? ras[i] : 0u;
       }
     }
#pragma unroll
     for (int j = 0; j < kBinLoads; ++j) {
      if (b + 32u * j >= n) break;  // warp-uniform
      unsigned key = ~0u;  // 2 cell + side, or none
      int kf = 0;
      unsigned long long res = 0;
      if (rcv[j] != ~0u) {
        const uint32_t rc = rcv[j];
        const int side = rc >> 31;
        const uint32_t cell = rc & 0x7FFFFFFFu;
        if constexpr (BATCH) tab[inst_of_cell(cell, nhi, mag)].of(rav[j], side, kf, res);
        else sh.of(rav[j], side, kf, res);
        key = 2u * cell + (unsigned)side;
      }
      const unsigned prev = __shfl_up_sync(0xFFFFFFFFu, key, 1);
      const bool head = lane == 0 || prev != key;
      const unsigned heads = __ballot_sync(0xFFFFFFFFu, head);
      const unsigned later = heads & ~((2u << lane) - 1u);
      const int end = later ? __ffs(later) - 1 : 32;  // the next run's first lane
      if (heads != 0xFFFFFFFFu) {  // some run is longer than one record
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const int kf2 = __shfl_down_sync(0xFFFFFFFFu, kf, off);
          const unsigned long long res2 = __shfl_down_sync(0xFFFFFFFFu, res, off);
          if (lane + off < end) {
            kf += kf2;
            res += res2;
          }
        }
      }
      if (head && key != ~0u) {
        const int side = key & 1u;
        const uint32_t cell = key >> 1;
        if (kf) atomicAdd((side ? keep1 : keep0) + cell, kf);
        if (res) atomicAdd((side ? res1 : res0) + cell, res);
        if constexpr (!BATCH) {
          if (side) ks1 += (unsigned long long)kf; else ks0 += (unsigned long long)kf;
        }
      }
     }
    }
  }
  if constexpr (!BATCH) {
    for (int s = 0; s < 2; ++s) {
      unsigned long long t;
      block_exscan(s ? ks1 : ks0, red, t);
      if (threadIdx.x == 0 && t) atomicAdd(&c->boot_keep[s], t);
    }
  }
}

// Guide table of the draws (the indexed search of Chen and Asau): for each
// side and bucket j of the top kGuideBits bits of r, G_j = the first cell
// whose inclusive residual prefix exceeds floor(j R / 2^kGuideBits), and
// G_{2^kGuideBits} = nh - 1.  A draw with r in bucket j has its cell in
// [G_j, G_{j+1}].
__global__ void __launch_bounds__(kBlock) k_boot_guide(const Counters* c, long long nh,
                                                       const unsigned long long* pre0,
                                                       const unsigned long long* pre1,
                                                       int* guide) {
  const int per = kGuide + 1;
  for (int i = blockIdx.x * kBlock + threadIdx.x; i < 2 * per; i += gridDim.x * kBlock) {
    const int side = i / per, j = i - side * per;
    const unsigned long long* pre = side ? pre1 : pre0;
    long long lo = 0, hi = nh - 1;
    if (j < kGuide) {
      const unsigned long long R = c->boot_R[side];
      const unsigned long long t = __umul64hi((unsigned long long)j << (64 - kGuideBits), R);
      while (lo < hi) {
        const long long mid = lo + (hi - lo) / 2;
        if (pre[mid] > t) hi = mid; else lo = mid + 1;
      }
    } else {
      lo = nh - 1;
    }
    guide[i] = (int)lo;
  }
}

// N_r^s = N^s - sum floor(q_i) draws per side, each an upper-bound search of
// U = floor(r R / 2^64) in the inclusive residual prefix, within the range
// the guide table gives.
__global__ void __launch_bounds__(kBlock) k_boot_draw(Counters* c, long long nh,
                                                      const unsigned long long* pre0,
                                                      const unsigned long long* pre1,
                                                      int* keep0, int* keep1,
                                                      const int* guide, uint32_t key0,
                                                      uint32_t key1, int epoch_delta) {
  const unsigned long long epoch = (c->per_regen_base >> 40) + (unsigned long long)epoch_delta;
  unsigned long long nr[2];
  for (int s = 0; s < 2; ++s) {
    const long long d = (long long)c->boot_n[s] - (long long)c->boot_keep[s];
    nr[s] = d > 0 ? (unsigned long long)d : 0ull;
    if (c->boot_R[s] == 0) nr[s] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->boot_nr[0] = nr[0];
    c->boot_nr[1] = nr[1];
  }
  const unsigned long long total = nr[0] + nr[1];
  for (unsigned long long i = (unsigned long long)blockIdx.x * kBlock + threadIdx.x; i < total;
       i += (unsigned long long)gridDim.x * kBlock) {
    const int side = i < nr[0] ? 0 : 1;
    const unsigned long long d = side ? i - nr[0] : i;
    const uint4 r = philox((uint32_t)d, (uint32_t)(d >> 32), kStepBoot,
                           (uint32_t)((epoch << 1) | (unsigned long long)side), key0, key1);
    const unsigned long long r64 = ((unsigned long long)r.y << 32) | r.x;
    const unsigned long long U = __umul64hi(r64, c->boot_R[side]);
    const unsigned long long* pre = side ? pre1 : pre0;
    const int* gs = guide + side * (kGuide + 1);
    const int j = (int)(r64 >> (64 - kGuideBits));
    int lo = gs[j], hi = gs[j + 1];  // first cell with pre > U (nh < 2^31)
    while (lo < hi) {
      const int mid = lo + ((hi - lo) >> 1);
      if (pre[mid] > U) hi = mid; else lo = mid + 1;
    }
    atomicAdd((side ? keep1 : keep0) + lo, 1);
  }
}

// m_nu = (W^+/N^+) n~+ - (W^-/N^-) n~- (= N_alpha mu d_nu), rounded as Alg. 3.
__global__ void __launch_bounds__(kBlock) k_boot_combine(const Counters* c, long long nh,
                                                         const int* keep0, const int* keep1,
                                                         int* grid, uint32_t key0,
                                                         uint32_t key1, int epoch_delta) {
  const unsigned long long epoch = (c->per_regen_base >> 40) + (unsigned long long)epoch_delta;
  double amp[2];
  for (int s = 0; s < 2; ++s)
    amp[s] = c->boot_n[s] > 0
                 ? __ddiv_rn(__dmul_rn((double)c->boot_w[s], 1.0 / 2147483648.0),
                             (double)c->boot_n[s])
                 : 0.0;
  for (long long nu = (long long)blockIdx.x * kBlock + threadIdx.x; nu < nh;
       nu += (long long)gridDim.x * kBlock) {
    const double m = __dsub_rn(__dmul_rn((double)keep0[nu], amp[0]),
                               __dmul_rn((double)keep1[nu], amp[1]));
    const double am = fabs(m);
    const double fl = floor(am);
    const uint4 r = philox((uint32_t)nu, (uint32_t)((unsigned long long)nu >> 32), kStepRound,
                           (uint32_t)epoch, key0, key1);
    const double u = u53(r.x, r.y);
    const long long cnt = (long long)fl + (u < __dsub_rn(am, fl) ? 1 : 0);
    grid[nu] = (int)(m < 0 ? -cnt : cnt);
  }
}

// ---------------------------------------------------------------------------
// sp2 in a batch: Alg. 2 per instance and side.  Instance b owns the global
// cells [b nhi, (b + 1) nhi); its draws and roundings are counted by
// (b << 32) | d and (b << 32) | (nu - b nhi), so that instance b is the run
// of salt b (a plain run is salt 0).
// ---------------------------------------------------------------------------

// Adds one run's counts and weight sums of instance i (both sides) to the
// shared per-instance sums.
__device__ __forceinline__ void flush_tally(unsigned long long* sn, unsigned long long* sw, int i,
                                            unsigned long long c0, unsigned long long c1,
                                            unsigned long long w0, unsigned long long w1) {
  if (c0) { atomicAdd(sn + 2 * i, c0); atomicAdd(sw + 2 * i, w0); }
  if (c1) { atomicAdd(sn + 2 * i + 1, c1); atomicAdd(sw + 2 * i + 1, w1); }
}

// N^s and W^s of every instance: its offspring records (cell | side << 31,
// a) and its unit-weight counts (a = 2^31 each), summed per block in shared
// memory and added to the instances' records.
__global__ void __launch_bounds__(kBlock, kTallyBlocks)
    k_bootb_tally(const uint32_t* rec_cell, const uint32_t* rec_a, const unsigned* rcnt, int nseg,
                  long long rseg, const int* ucnt, long long nh, int nhi, int ninst,
                  BootInst* bi) {
  const unsigned long long mag = inst_magic(nhi);
  __shared__ unsigned long long sn[2 * kMaxInst], sw[2 * kMaxInst];
  for (int i = threadIdx.x; i < 2 * ninst; i += kBlock) sn[i] = sw[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * kBlock + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * kBlock) >> 5;
  const long long cps = (rseg + kBootChunk - 1) / kBootChunk;
  for (long long it = gw; it < (long long)nseg * cps; it += nw) {
    const long long sg = it / cps;
    const unsigned b0 = (unsigned)((it - sg * cps) * kBootChunk);
    const unsigned n = min(min(rcnt[sg], (unsigned)rseg), b0 + (unsigned)kBootChunk);
    // a segment holds runs of one instance's records (of both signs, the
    // pairs interleaved)
    const uint32_t* rcs = rec_cell + sg * rseg;
    const uint32_t* ras = rec_a + sg * rseg;
    // kTallyLoads groups of 32 records are loaded before the first is used,
    // so that each warp keeps that many loads in flight (the kernel streams
    // the records once).  While consecutive groups belong to one instance
    // their sums stay in registers (the same in every lane); they go to the
    // block's shared sums when another instance's group comes and at the end
    // of the chunk.
    int cur = -1;
    unsigned rc0 = 0, rc1 = 0;
    unsigned long long rw0 = 0, rw1 = 0;
    for (unsigned b = b0; b < n; b += 32u * kTallyLoads) {
      uint32_t rcv[kTallyLoads], rav[kTallyLoads];
#pragma unroll
      for (int j = 0; j < kTallyLoads; ++j) {
        const unsigned i = b + 32u * j + lane;
        rcv[j] = i < n ? __ldcs(rcs + i) : ~0u;
        rav[j] = i < n ? __ldcs(ras + i) : 0u;
      }
#pragma unroll
      for (int j = 0; j < kTallyLoads; ++j) {
        if (b + 32u * j >= n) break;  // warp-uniform: lane 0's record exists below
        const bool valid = rcv[j] != ~0u;
        const int side = (int)(rcv[j] >> 31);
        const int inst = valid ? (int)inst_of_cell(rcv[j] & 0x7FFFFFFFu, nhi, mag) : -1;
        const unsigned a = rav[j];
        const int inst0 = __shfl_sync(0xFFFFFFFFu, inst, 0);
        if (__all_sync(0xFFFFFFFFu, inst == inst0 || inst < 0)) {
          // the warp's records belong to one instance: counts by ballots,
          // weight sums in 16-bit halves
          const bool s0 = valid && side == 0, s1 = valid && side == 1;
          const unsigned c0 = __popc(__ballot_sync(0xFFFFFFFFu, s0));
          const unsigned c1 = __popc(__ballot_sync(0xFFFFFFFFu, s1));
          const unsigned lo0 = __reduce_add_sync(0xFFFFFFFFu, s0 ? a & 0xFFFFu : 0u);
          const unsigned hi0 = __reduce_add_sync(0xFFFFFFFFu, s0 ? a >> 16 : 0u);
          const unsigned lo1 = __reduce_add_sync(0xFFFFFFFFu, s1 ? a & 0xFFFFu : 0u);
          const unsigned hi1 = __reduce_add_sync(0xFFFFFFFFu, s1 ? a >> 16 : 0u);
          const unsigned long long w0 = ((unsigned long long)hi0 << 16) + lo0;
          const unsigned long long w1 = ((unsigned long long)hi1 << 16) + lo1;
          if (inst0 != cur) {  // a new run: the last one to the shared sums
            if (lane == 0 && cur >= 0) flush_tally(sn, sw, cur, rc0, rc1, rw0, rw1);
            cur = inst0;
            rc0 = rc1 = 0;
            rw0 = rw1 = 0;
          }
          rc0 += c0;
          rc1 += c1;
          rw0 += w0;
          rw1 += w1;
          continue;
        }
        // mixed instances: runs of equal instances in consecutive lanes, each
        // run's first lane adding the run's sums
        unsigned c0 = valid && side == 0, c1 = valid && side == 1;
        unsigned long long w0 = c0 ? a : 0ull, w1 = c1 ? a : 0ull;
        const int prev = __shfl_up_sync(0xFFFFFFFFu, inst, 1);
        const bool head = lane == 0 || prev != inst;
        const unsigned heads = __ballot_sync(0xFFFFFFFFu, head);
        const unsigned later = heads & ~((2u << lane) - 1u);
        const int end = later ? __ffs(later) - 1 : 32;  // the next run's first lane
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const unsigned d0 = __shfl_down_sync(0xFFFFFFFFu, c0, off);
          const unsigned d1 = __shfl_down_sync(0xFFFFFFFFu, c1, off);
          const unsigned long long v0 = __shfl_down_sync(0xFFFFFFFFu, w0, off);
          const unsigned long long v1 = __shfl_down_sync(0xFFFFFFFFu, w1, off);
          if (lane + off < end) {
            c0 += d0;
            c1 += d1;
            w0 += v0;
            w1 += v1;
          }
        }
        if (head && inst >= 0) flush_tally(sn, sw, inst, c0, c1, w0, w1);
      }
    }
    if (lane == 0 && cur >= 0) flush_tally(sn, sw, cur, rc0, rc1, rw0, rw1);
  }
  // unit counts: warps over consecutive cells
  for (long long c0 = gw * 32; c0 < nh; c0 += nw * 32) {
    const long long nu = c0 + lane;
    const int inst = nu < nh ? (int)inst_of_cell((unsigned)nu, nhi, mag) : -1;
    for (int sd = 0; sd < 2; ++sd) {
      const unsigned u = nu < nh ? (unsigned)ucnt[sd * nh + nu] : 0u;
      const int key = inst < 0 || u == 0 ? -1 : 2 * inst + sd;
      // the count once, the weight (u 2^31 each) from the count
      const unsigned grp = __match_any_sync(0xFFFFFFFFu, key);
      if (key >= 0) {
        const unsigned t = __reduce_add_sync(grp, u);
        if (lane == __ffs(grp) - 1) {
          atomicAdd(sn + key, (unsigned long long)t);
          atomicAdd(sw + key, (unsigned long long)t << 31);
        }
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * ninst; i += kBlock) {
    if (sn[i]) atomicAdd(&bi[i >> 1].n[i & 1], sn[i]);
    if (sw[i]) atomicAdd(&bi[i >> 1].w[i & 1], sw[i]);
  }
}

// Each instance's shares (BootShare from its N^s, W^s), the share of a unit
// weight and the amplitudes of the combination step.
__global__ void __launch_bounds__(kBlock) k_bootb_share(BootInst* bi, int ninst, int fx) {
  for (int i = blockIdx.x * kBlock + threadIdx.x; i < ninst; i += gridDim.x * kBlock) {
    BootInst& b = bi[i];
    BootShare sh;
    sh.init(b.n, b.w, fx);
    b.ratio[0] = sh.ratio0;
    b.ratio[1] = sh.ratio1;
    b.mx[0] = sh.mx0;
    b.mx[1] = sh.mx1;
    b.fx[0] = sh.fx0;
    b.fx[1] = sh.fx1;
    for (int sd = 0; sd < 2; ++sd) {
      int kf;
      unsigned long long rs;
      sh.of(2147483648u, sd, kf, rs);
      b.kf_unit[sd] = kf;
      b.res_unit[sd] = rs;
      b.amp[sd] = b.n[sd] > 0 ? __ddiv_rn(__dmul_rn((double)b.w[sd], 1.0 / 2147483648.0),
                                          (double)b.n[sd])
                              : 0.0;
    }
  }
}

// The unit-weight part of every cell (k_boot_unit per instance).
__global__ void __launch_bounds__(kBlock) k_bootb_unit(const BootInst* bi, const int* ucnt,
                                                       long long nh, int nhi, int* keep0,
                                                       int* keep1, unsigned long long* res0,
                                                       unsigned long long* res1) {
  const unsigned long long mag = inst_magic(nhi);
  for (long long nu = (long long)blockIdx.x * kBlock + threadIdx.x; nu < nh;
       nu += (long long)gridDim.x * kBlock) {
    const BootInst& b = bi[inst_of_cell((unsigned)nu, nhi, mag)];
    const int u0 = ucnt[nu], u1 = ucnt[nh + nu];
    keep0[nu] = u0 * b.kf_unit[0];
    keep1[nu] = u1 * b.kf_unit[1];
    res0[nu] = (unsigned long long)u0 * b.res_unit[0];
    res1[nu] = (unsigned long long)u1 * b.res_unit[1];
  }
}

// Each instance's sums of the kept integer parts, over its cells (a warp's
// cells belong to one instance but at instance boundaries: the warp keeps
// the running sums of its current instance, as k_bootb_tally does).
__global__ void __launch_bounds__(kBlock) k_bootb_keep(BootInst* bi, const int* keep0,
                                                       const int* keep1, long long nh, int nhi) {
  const unsigned long long mag = inst_magic(nhi);
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * kBlock + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * kBlock) >> 5;
  int ci = -1;
  unsigned long long k0s = 0, k1s = 0;
  auto flush = [&]() {
    if (lane == 0 && ci >= 0) {
      if (k0s) atomicAdd(&bi[ci].keep[0], k0s);
      if (k1s) atomicAdd(&bi[ci].keep[1], k1s);
    }
    k0s = k1s = 0;
  };
  for (long long c0 = gw * 32; c0 < nh; c0 += nw * 32) {
    const long long nu = c0 + lane;
    const int inst = nu < nh ? (int)inst_of_cell((unsigned)nu, nhi, mag) : -1;
    const unsigned k0 = nu < nh ? (unsigned)keep0[nu] : 0u;
    const unsigned k1 = nu < nh ? (unsigned)keep1[nu] : 0u;
    const int inst0 = __shfl_sync(0xFFFFFFFFu, inst, 0);
    if (__all_sync(0xFFFFFFFFu, inst == inst0 || inst < 0)) {
      // 32 kept counts of 32-bit cells: the sums taken in 16-bit halves
      const unsigned long long t0 =
          ((unsigned long long)__reduce_add_sync(0xFFFFFFFFu, k0 >> 16) << 16) +
          __reduce_add_sync(0xFFFFFFFFu, k0 & 0xFFFFu);
      const unsigned long long t1 =
          ((unsigned long long)__reduce_add_sync(0xFFFFFFFFu, k1 >> 16) << 16) +
          __reduce_add_sync(0xFFFFFFFFu, k1 & 0xFFFFu);
      if (t0 | t1) {
        if (inst0 != ci) {
          flush();
          ci = inst0;
        }
        k0s += t0;
        k1s += t1;
      }
    } else if (inst >= 0) {  // an instance boundary inside the warp
      if (k0) atomicAdd(&bi[inst].keep[0], (unsigned long long)k0);
      if (k1) atomicAdd(&bi[inst].keep[1], (unsigned long long)k1);
    }
  }
  flush();
}

// Per instance and side: the residual total R (from the inclusive prefix
// over all cells), N_r = N - sum floor(q) draws (none without a residual),
// and the exclusive prefix of the draws over (instance, side) pairs; the
// run's counters get the totals.  One block.
__global__ void __launch_bounds__(kBlock) k_bootb_plan(Counters* c, BootInst* bi,
                                                       const unsigned long long* pre0,
                                                       const unsigned long long* pre1,
                                                       int ninst, int nhi,
                                                       unsigned long long* dpre) {
  static_assert(kMaxInst <= kBlock, "one thread per instance");
  __shared__ unsigned long long red[kBlock / 32 + 1];
  const int i = threadIdx.x;  // ninst <= kBlock
  unsigned long long nr[2] = {0, 0};
  if (i < ninst) {
    BootInst& b = bi[i];
    const long long first = (long long)i * nhi, last = first + nhi - 1;
    for (int sd = 0; sd < 2; ++sd) {
      const unsigned long long* pre = sd ? pre1 : pre0;
      const unsigned long long base = first > 0 ? pre[first - 1] : 0ull;
      const unsigned long long R = pre[last] - base;
      b.base[sd] = base;
      b.R[sd] = R;
      nr[sd] = (R > 0 && b.n[sd] > b.keep[sd]) ? b.n[sd] - b.keep[sd] : 0ull;
      b.nr[sd] = nr[sd];
    }
  }
  unsigned long long total;
  const unsigned long long ex = block_exscan(nr[0] + nr[1], red, total);
  if (i < ninst) {
    dpre[2 * i] = ex;
    dpre[2 * i + 1] = ex + nr[0];
  }
  if (i == 0) {
    dpre[2 * ninst] = total;
    for (int sd = 0; sd < 2; ++sd) {
      unsigned long long k = 0, r = 0, R = 0;
      for (int j = 0; j < ninst; ++j) {
        k += bi[j].keep[sd];
        r += bi[j].nr[sd];
        R += bi[j].R[sd];
      }
      c->boot_keep[sd] = k;
      c->boot_nr[sd] = r;
      c->boot_R[sd] = R;
    }
  }
}

// Guide tables of the draws per instance and side (k_boot_guide's, on the
// instance's cells and its prefix less base): G_j = the first cell of the
// instance whose prefix exceeds floor(j R / 2^kGuideBitsB), G_last = the
// instance's last cell.
__global__ void __launch_bounds__(kBlock) k_bootb_guide(const BootInst* bi,
                                                        const unsigned long long* pre0,
                                                        const unsigned long long* pre1,
                                                        int ninst, int nhi, int* guide) {
  const int per = kGuideB + 1;
  for (long long t = (long long)blockIdx.x * kBlock + threadIdx.x; t < 2ll * ninst * per;
       t += (long long)gridDim.x * kBlock) {
    const int pair = (int)(t / per), j = (int)(t - (long long)pair * per);
    const int inst = pair >> 1, side = pair & 1;
    const BootInst& b = bi[inst];
    int lo = inst * nhi, hi = lo + nhi - 1;
    if (j < kGuideB && b.nr[side] > 0) {
      const unsigned long long th =
          __umul64hi((unsigned long long)j << (64 - kGuideBitsB), b.R[side]) + b.base[side];
      const unsigned long long* pre = side ? pre1 : pre0;
      while (lo < hi) {
        const int mid = lo + ((hi - lo) >> 1);
        if (pre[mid] > th) hi = mid; else lo = mid + 1;
      }
    } else {
      lo = hi;
    }
    guide[t] = lo;
  }
}

// The residual draws of all instances: draw i belongs to the (instance,
// side) pair whose prefix range holds it and is that pair's draw d; its cell
// is the first of the instance whose residual prefix (less base) exceeds
// U = floor(r R / 2^64).
__global__ void __launch_bounds__(kBlock) k_bootb_draw(
    const Counters* c, const BootInst* bi, const unsigned long long* dpre,
    const unsigned long long* pre0, const unsigned long long* pre1, int ninst, int nhi,
    const int* guide, int* keep0, int* keep1, uint32_t key0, uint32_t key1, int epoch_delta) {
  __shared__ unsigned long long sp[2 * kMaxInst + 1];
  const int np = 2 * ninst;
  for (int i = threadIdx.x; i <= np; i += kBlock) sp[i] = dpre[i];
  __syncthreads();
  const unsigned long long epoch = (c->per_regen_base >> 40) + (unsigned long long)epoch_delta;
  const unsigned long long total = sp[np];
  for (unsigned long long i = (unsigned long long)blockIdx.x * kBlock + threadIdx.x; i < total;
       i += (unsigned long long)gridDim.x * kBlock) {
    int a = 0, z = np;  // the pair with sp[a] <= i < sp[a + 1]
    while (z - a > 1) {
      const int m = (a + z) >> 1;
      if (sp[m] <= i) a = m; else z = m;
    }
    const int inst = a >> 1, side = a & 1;
    const unsigned long long d = i - sp[a];
    const uint4 r = philox((uint32_t)d, (uint32_t)inst, kStepBoot,
                           (uint32_t)((epoch << 1) | (unsigned long long)side), key0, key1);
    const unsigned long long r64 = ((unsigned long long)r.y << 32) | r.x;
    const BootInst& b = bi[inst];
    // U + base < the prefix at the instance's last cell
    const unsigned long long U = __umul64hi(r64, b.R[side]) + b.base[side];
    const unsigned long long* pre = side ? pre1 : pre0;
    const int* gs = guide + (size_t)a * (kGuideB + 1);
    const int j = (int)(r64 >> (64 - kGuideBitsB));
    int lo = gs[j], hi = gs[j + 1];  // the cell lies in [G_j, G_{j+1}]
    while (lo < hi) {
      const int mid = lo + ((hi - lo) >> 1);
      if (pre[mid] > U) hi = mid; else lo = mid + 1;
    }
    atomicAdd((side ? keep1 : keep0) + lo, 1);
  }
}

// k_boot_combine per instance: the amplitudes of the cell's instance and the
// rounding counted by (instance << 32) | (cell within the instance).
__global__ void __launch_bounds__(kBlock) k_bootb_combine(const Counters* c, const BootInst* bi,
                                                          long long nh, int nhi,
                                                          const int* keep0, const int* keep1,
                                                          int* grid, uint32_t key0,
                                                          uint32_t key1, int epoch_delta) {
  const unsigned long long mag = inst_magic(nhi);
  const unsigned long long epoch = (c->per_regen_base >> 40) + (unsigned long long)epoch_delta;
  for (long long nu = (long long)blockIdx.x * kBlock + threadIdx.x; nu < nh;
       nu += (long long)gridDim.x * kBlock) {
    const int inst = (int)inst_of_cell((unsigned)nu, nhi, mag);  // nh < 2^30
    const BootInst& b = bi[inst];
    const double m = __dsub_rn(__dmul_rn((double)keep0[nu], b.amp[0]),
                               __dmul_rn((double)keep1[nu], b.amp[1]));
    const double am = fabs(m);
    const double fl = floor(am);
    const uint4 r = philox((uint32_t)(nu - (long long)inst * nhi), (uint32_t)inst, kStepRound,
                           (uint32_t)epoch, key0, key1);
    const double u = u53(r.x, r.y);
    const long long cnt = (long long)fl + (u < __dsub_rn(am, fl) ? 1 : 0);
    grid[nu] = (int)(m < 0 ? -cnt : cnt);
  }
}

// wp: the weighted histogram (Eq. piecewise_constant_function, weights in
// fixed point 2^-31) rounded by Alg. 3: floor(|m|) particles plus one with
// probability |m| - floor(|m|), sign of m, the uniform of the draw
// ((b << 32) | cell within instance b, ROUND, epoch) as for sp2 (b = 0 in a
// plain run).
__global__ void __launch_bounds__(kBlock) k_wp_round(const Counters* c, long long nh, int nhi,
                                                     const long long* wsum, int* grid,
                                                     uint32_t key0, uint32_t key1,
                                                     int epoch_delta) {
  const unsigned long long mag = inst_magic(nhi);
  const unsigned long long epoch = (c->per_regen_base >> 40) + (unsigned long long)epoch_delta;
  for (long long nu = (long long)blockIdx.x * kBlock + threadIdx.x; nu < nh;
       nu += (long long)gridDim.x * kBlock) {
    const double m = __dmul_rn((double)wsum[nu], 1.0 / 2147483648.0);
    const double am = fabs(m);
    const double fl = floor(am);
    const int inst = (int)inst_of_cell((unsigned)nu, nhi, mag);  // nh < 2^30
    const uint4 r = philox((uint32_t)(nu - (long long)inst * nhi), (uint32_t)inst, kStepRound,
                           (uint32_t)epoch, key0, key1);
    const double u = u53(r.x, r.y);
    const long long cnt = (long long)fl + (u < __dsub_rn(am, fl) ? 1 : 0);
    grid[nu] = (int)(m < 0 ? -cnt : cnt);
  }
}

// ---------------------------------------------------------------------------
// Observables: one warp per x-column.
// ---------------------------------------------------------------------------
// counts (int) or wsum (int64, each value times scale) per cell, x-major.
__global__ void __launch_bounds__(kBlock) k_obs_cols(const int* counts, const long long* wsum,
                                                     int nx, int nk, double na, double dx,
                                                     double dk, double scale, double* density,
                                                     double* marg, long long* col) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * kBlock + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * kBlock) >> 5;
  for (long long ix = warp; ix < nx; ix += nwarps) {
    long long s = 0;
    for (int ik = lane; ik < nk; ik += 32) {
      const long long nu = ix * nk + ik;
      const long long v = wsum ? wsum[nu] : (long long)counts[nu];
      s += v;
      if (density)
        density[nu] = __ddiv_rn(__dmul_rn((double)v, scale), __dmul_rn(__dmul_rn(na, dx), dk));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
    if (lane == 0) {
      col[ix] = s;
      marg[ix] = __ddiv_rn(__dmul_rn((double)s, scale), __dmul_rn(na, dx));
    }
  }
}

__global__ void __launch_bounds__(kBlock) k_obs_total(const long long* col, int nx, double xmin,
                                                      double dx, double na, double scale,
                                                      double* out) {
  __shared__ unsigned long long red[kBlock / 32 + 1];
  long long s = 0;
  for (int ix = threadIdx.x; ix < nx; ix += kBlock) {
    const double centre = __dadd_rn(xmin, __dmul_rn(__dadd_rn((double)ix, 0.5), dx));
    if (centre > 0.0) s += col[ix];
  }
  unsigned long long t;
  block_exscan((unsigned long long)s, red, t);
  if (threadIdx.x == 0)
    out[0] = __ddiv_rn(__dmul_rn((double)(long long)t, scale), na);
}

// Transmission of each instance (one block each): the sum of its counts
// over the cells with centre x > 0, divided by its N_alpha.  The cells with
// centre x > 0 are the columns ix >= ix0, a contiguous range.
__global__ void __launch_bounds__(kBlock) k_obs_trans(const int* counts, int nx, int nk,
                                                      double xmin, double dx, const double* na,
                                                      double* out) {
  __shared__ unsigned long long red[kBlock / 32 + 1];
  __shared__ int s_ix0;
  if (threadIdx.x == 0) {
    int ix0 = nx;
    for (int ix = 0; ix < nx; ++ix)
      if (__dadd_rn(xmin, __dmul_rn(__dadd_rn((double)ix, 0.5), dx)) > 0.0) { ix0 = ix; break; }
    s_ix0 = ix0;
  }
  __syncthreads();
  const long long nhi = (long long)nx * nk;
  const int* g = counts + (long long)blockIdx.x * nhi;
  long long s = 0;
  for (long long nu = (long long)s_ix0 * nk + threadIdx.x; nu < nhi; nu += kBlock) s += g[nu];
  unsigned long long t;
  block_exscan((unsigned long long)s, red, t);
  if (threadIdx.x == 0) out[blockIdx.x] = __ddiv_rn((double)(long long)t, na[blockIdx.x]);
}

// Particles of one instance in the arrays: its base slots plus the offspring
// labelled with it.
__global__ void __launch_bounds__(kBlock) k_live_inst(const Counters* c,
                                                      const unsigned long long* inst_slot,
                                                      const unsigned* cinst, int inst,
                                                      unsigned long long* out) {
  __shared__ unsigned long long red[kBlock / 32 + 1];
  const unsigned long long n = c->n, nb = c->n_base;
  unsigned long long s = 0;
  for (unsigned long long i = nb + (unsigned long long)blockIdx.x * kBlock + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * kBlock)
    s += cinst[i - nb] == (unsigned)inst;
  if (blockIdx.x == 0 && threadIdx.x == 0) s += inst_slot[inst + 1] - inst_slot[inst];
  unsigned long long t;
  block_exscan(s, red, t);
  if (threadIdx.x == 0 && t) atomicAdd(out, t);
}

// The 4D counts summed over electron 2: red[ix1 nk + ik1] =
// sum over (ix2, ik2) of counts[((ix1 nx + ix2) nk + ik1) nk + ik2], one warp
// per output.
__global__ void __launch_bounds__(kBlock) k_reduce4(const int* counts, int nx, int nk,
                                                    long long* red) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * kBlock + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * kBlock) >> 5;
  for (long long o = warp; o < (long long)nx * nk; o += nwarps) {
    const long long ix1 = o / nk, ik1 = o % nk;
    long long s = 0;
    for (long long ix2 = 0; ix2 < nx; ++ix2) {
      const int* row = counts + ((ix1 * nx + ix2) * nk + ik1) * nk;
      for (int ik2 = lane; ik2 < nk; ik2 += 32) s += row[ik2];
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, d);
    if (lane == 0) red[o] = s;
  }
}

// ---------------------------------------------------------------------------
// Tangent plan (tangent mode): cell nu carries n_nu = ceil(max(|D_H|, |D_w|)
// / quantum) tangent particles with tau = D_nu / n_nu each.  The same three
// passes as the plan of the signed particles.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long tan_count(const long long* dH, const long long* dw,
                                                       long long c, long long q) {
  const long long a = dH[c] < 0 ? -dH[c] : dH[c], b = dw[c] < 0 ? -dw[c] : dw[c];
  const long long m = a > b ? a : b;
  return m ? (unsigned long long)((m + q - 1) / q) : 0ull;
}

__global__ void __launch_bounds__(kBlock) k_tcells_a(const long long* dH, const long long* dw,
                                                     long long nh, long long q,
                                                     unsigned long long* bsum, unsigned int* bnz) {
  __shared__ unsigned long long red[kBlock / 32 + 1];
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  unsigned long long s = 0, z = 0;
  for (int i = 0; i < kScanItems; ++i) {
    const long long c = base + i;
    if (c < nh) {
      const unsigned long long n = tan_count(dH, dw, c, q);
      s += n;
      z += n != 0;
    }
  }
  unsigned long long ts, tz;
  block_exscan(s, red, ts);
  block_exscan(z, red, tz);
  if (threadIdx.x == 0) {
    bsum[blockIdx.x] = ts;
    bnz[blockIdx.x] = (unsigned int)tz;
  }
}

__global__ void __launch_bounds__(kBlock) k_tcells_c(const long long* dH, const long long* dw,
                                                     long long nh, long long q,
                                                     const unsigned long long* bsum,
                                                     const unsigned int* bnz, uint32_t* nz_cell,
                                                     unsigned long long* nz_start, double* nz_tau,
                                                     uint32_t* tile_nz, long long tile_cap,
                                                     long long nhi, unsigned long long* inst_slot) {
  __shared__ unsigned long long red[kBlock / 32 + 1];
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  unsigned long long n[kScanItems];  // unrolled loops keep it in registers
  unsigned long long s = 0, z = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const long long c = base + i;
    n[i] = c < nh ? tan_count(dH, dw, c, q) : 0ull;
    s += n[i];
    z += n[i] != 0;
  }
  unsigned long long ts, tz;
  unsigned long long os = block_exscan(s, red, ts) + bsum[blockIdx.x];
  unsigned long long oz = block_exscan(z, red, tz) + bnz[blockIdx.x];
  long long next_inst = (base + nhi - 1) / nhi * nhi;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const long long c = base + i;
    if (c == next_inst && next_inst < nh) {
      inst_slot[next_inst / nhi] = os;
      next_inst += nhi;
    }
    if (n[i]) {
      nz_cell[oz] = (uint32_t)c;
      nz_start[oz] = os;
      nz_tau[2 * oz] = __ddiv_rn(__dmul_rn((double)dH[c], 1.0 / 4294967296.0), (double)n[i]);
      nz_tau[2 * oz + 1] = __ddiv_rn(__dmul_rn((double)dw[c], 1.0 / 4294967296.0), (double)n[i]);
      const unsigned long long t_end = min((os + n[i] + 31) >> 5, (unsigned long long)tile_cap);
      for (unsigned long long t = (os + 31) >> 5; t < t_end; ++t) tile_nz[t] = (uint32_t)oz;
      ++oz;
      os += n[i];
    }
  }
}

// (dT/dH, dT/dw) of each instance (one block each): the tangent histogram
// summed over the cells with centre x > 0, times 2^-32, over N_alpha.
__global__ void __launch_bounds__(kBlock) k_obs_tgrad(const long long* dH, const long long* dw,
                                                      int nx, int nk, double xmin, double dx,
                                                      const double* na, double* out) {
  __shared__ unsigned long long red[kBlock / 32 + 1];
  __shared__ int s_ix0;
  if (threadIdx.x == 0) {
    int ix0 = nx;
    for (int ix = 0; ix < nx; ++ix)
      if (__dadd_rn(xmin, __dmul_rn(__dadd_rn((double)ix, 0.5), dx)) > 0.0) { ix0 = ix; break; }
    s_ix0 = ix0;
  }
  __syncthreads();
  const long long nhi = (long long)nx * nk;
  for (int d = 0; d < 2; ++d) {
    const long long* g = (d ? dw : dH) + (long long)blockIdx.x * nhi;
    long long acc = 0;
    for (long long nu = (long long)s_ix0 * nk + threadIdx.x; nu < nhi; nu += kBlock) acc += g[nu];
    unsigned long long t;
    block_exscan((unsigned long long)acc, red, t);
    if (threadIdx.x == 0)
      out[2 * blockIdx.x + d] =
          __ddiv_rn(__dmul_rn((double)(long long)t, 1.0 / 4294967296.0), na[blockIdx.x]);
    __syncthreads();
  }
}

int grid_cap(Ctx* c, int per_sm) { return c->num_sms * per_sm; }

}  // namespace

cudaError_t launch_setup(Ctx* c, int op, unsigned long long a, unsigned long long b) {
  if (op == SETUP_CHUNK || op == SETUP_AFTER_REGEN) c->dev_period_ok = 0;
  if (op == SETUP_PERIOD) c->dev_period_ok = 1;
  k_setup<<<1, 32, 0, c->stream>>>(c->cnt, op, a, b);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_zero(Ctx* c, void* p, size_t bytes) {
  return cudaMemsetAsync(p, 0, bytes, c->stream);
}

cudaError_t launch_scan_cells(Ctx* c, const int* grid) {
  const long long nb = c->scan_blocks;
  k_cells_a<<<(unsigned)nb, kBlock, 0, c->stream>>>(grid, c->nh, c->scan_bsum, c->scan_bnz);
  k_cells_b<<<1, kBlock, 0, c->stream>>>(c->scan_bsum, c->scan_bnz, nb, c->cnt, c->tile_cap,
                                         c->inst_slot + c->ninst, 0);
  k_cells_c<<<(unsigned)nb, kBlock, 0, c->stream>>>(grid, c->nh, c->scan_bsum, c->scan_bnz,
                                                   c->nz_cell, c->nz_start, c->tile_nz,
                                                   c->tile_cap, c->nhi, c->inst_slot);
  c->launches += 3;
  return cudaGetLastError();
}

// sp2 in a batch: every instance bootstrapped on its own (Alg. 2 per
// instance and side), in the same launches.
static cudaError_t launch_boot_batch(Ctx* c, int epoch_delta) {
  const long long nh = c->nh, nb = c->scan_blocks;
  const int ni = c->ninst, nhi = (int)c->nhi;
  const uint32_t key0 = (uint32_t)c->cfg.seed, key1 = (uint32_t)(c->cfg.seed >> 32);
  const int fx = c->cfg.precision == WBRW_FP32;
  cudaError_t e = launch_zero(c, c->boot_inst, (size_t)ni * sizeof(BootInst));
  if (e != cudaSuccess) return e;
  k_bootb_tally<<<grid_cap(c, kTallyBlocks), kBlock, 0, c->stream>>>(
      c->rec_cell, c->rec_a, c->rcnt, c->nseg, c->rseg, c->boot_ucnt, nh, nhi, ni, c->boot_inst);
  k_bootb_share<<<1, kBlock, 0, c->stream>>>(c->boot_inst, ni, fx);
  k_bootb_unit<<<grid_cap(c, 8), kBlock, 0, c->stream>>>(c->boot_inst, c->boot_ucnt, nh, nhi,
                                                         c->boot_keep[0], c->boot_keep[1],
                                                         c->boot_res[0], c->boot_res[1]);
  k_boot_bin<true><<<grid_cap(c, kBootBinBatchBlocks), kBlock, 0, c->stream>>>(
      c->cnt, c->rec_cell, c->rec_a, c->rcnt, c->nseg, c->rseg, c->boot_keep[0], c->boot_keep[1],
      c->boot_res[0], c->boot_res[1], fx, c->boot_inst, ni, nhi);
  k_bootb_keep<<<grid_cap(c, 4), kBlock, 0, c->stream>>>(c->boot_inst, c->boot_keep[0],
                                                         c->boot_keep[1], nh, nhi);
  c->launches += 5;
  for (int s = 0; s < 2; ++s) {
    k_u64_a<<<(unsigned)nb, kBlock, 0, c->stream>>>(c->boot_res[s], nh, c->scan_bsum);
    k_u64_b<<<1, kBlock, 0, c->stream>>>(c->scan_bsum, nb, &c->cnt->boot_R[s]);
    k_u64_c<<<(unsigned)nb, kBlock, 0, c->stream>>>(c->boot_res[s], nh, c->scan_bsum);
    c->launches += 3;
  }
  k_bootb_plan<<<1, kBlock, 0, c->stream>>>(c->cnt, c->boot_inst, c->boot_res[0], c->boot_res[1],
                                            ni, nhi, c->boot_dpre);
  c->launches++;
  const long long ng = 2ll * ni * (kGuideB + 1);
  k_bootb_guide<<<(unsigned)((ng + kBlock - 1) / kBlock), kBlock, 0, c->stream>>>(
      c->boot_inst, c->boot_res[0], c->boot_res[1], ni, nhi, c->boot_bguide);
  k_bootb_draw<<<grid_cap(c, 8), kBlock, 0, c->stream>>>(
      c->cnt, c->boot_inst, c->boot_dpre, c->boot_res[0], c->boot_res[1], ni, nhi,
      c->boot_bguide, c->boot_keep[0], c->boot_keep[1], key0, key1, epoch_delta);
  k_bootb_combine<<<grid_cap(c, 8), kBlock, 0, c->stream>>>(c->cnt, c->boot_inst, nh, nhi,
                                                            c->boot_keep[0], c->boot_keep[1],
                                                            c->buf.grid, key0, key1, epoch_delta);
  c->launches += 3;
  return cudaGetLastError();
}

// Called after the records of the period are written and tallied.
// The resampling kernels read the epoch of the histogram they make from the
// device period state (the id base of the particles just binned, plus
// epoch_delta), so that a captured period replays with the right streams.
cudaError_t launch_boot(Ctx* c, int epoch_delta) {
  if (c->ninst > 1) return launch_boot_batch(c, epoch_delta);
  const long long nh = c->nh, nb = c->scan_blocks;
  const uint32_t key0 = (uint32_t)c->cfg.seed, key1 = (uint32_t)(c->cfg.seed >> 32);
  const int g = grid_cap(c, 8);
  const int fx = c->cfg.precision == WBRW_FP32;
  k_boot_unit<<<grid_cap(c, 4), kBlock, 0, c->stream>>>(c->cnt, c->boot_ucnt, nh, c->boot_keep[0],
                                                        c->boot_keep[1], c->boot_res[0],
                                                        c->boot_res[1], fx);
  c->launches++;
  k_boot_bin<false><<<grid_cap(c, kBootBinBlocks), kBlock, 0, c->stream>>>(
      c->cnt, c->rec_cell, c->rec_a, c->rcnt, c->nseg, c->rseg, c->boot_keep[0], c->boot_keep[1],
      c->boot_res[0], c->boot_res[1], fx, nullptr, 1, (int)c->nhi);
  c->launches++;
  for (int s = 0; s < 2; ++s) {
    k_u64_a<<<(unsigned)nb, kBlock, 0, c->stream>>>(c->boot_res[s], nh, c->scan_bsum);
    k_u64_b<<<1, kBlock, 0, c->stream>>>(c->scan_bsum, nb, &c->cnt->boot_R[s]);
    k_u64_c<<<(unsigned)nb, kBlock, 0, c->stream>>>(c->boot_res[s], nh, c->scan_bsum);
    c->launches += 3;
  }
  k_boot_guide<<<(2 * (kGuide + 1) + kBlock - 1) / kBlock, kBlock, 0, c->stream>>>(
      c->cnt, nh, c->boot_res[0], c->boot_res[1], c->boot_guide);
  k_boot_draw<<<g, kBlock, 0, c->stream>>>(
      c->cnt, nh, c->boot_res[0], c->boot_res[1], c->boot_keep[0], c->boot_keep[1], c->boot_guide,
      key0, key1, epoch_delta);
  k_boot_combine<<<g, kBlock, 0, c->stream>>>(c->cnt, nh, c->boot_keep[0], c->boot_keep[1],
                                              c->buf.grid, key0, key1, epoch_delta);
  c->launches += 3;
  return cudaGetLastError();
}

cudaError_t launch_wp_round(Ctx* c, int epoch_delta) {
  const uint32_t key0 = (uint32_t)c->cfg.seed, key1 = (uint32_t)(c->cfg.seed >> 32);
  k_wp_round<<<grid_cap(c, 8), kBlock, 0, c->stream>>>(c->cnt, c->nh, (int)c->nhi, c->tmp_wsum,
                                                       c->buf.grid, key0, key1, epoch_delta);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_observables(Ctx* c, int inst, const int* counts, const long long* wsum) {
  const double na = (double)c->ih[inst].n_alpha;
  const int g = grid_cap(c, 4);
  const long long off = (long long)inst * c->nhi;
  const int* cn = counts ? counts + off : nullptr;
  const long long* ws = wsum ? wsum + off : nullptr;
  double scale = wsum ? 1.0 / 2147483648.0 : 1.0;
  if (c->dim == 4 && cn) {  // electron 1's reduced counts
    k_reduce4<<<g, kBlock, 0, c->stream>>>(cn, c->cfg.nx, c->cfg.nk, c->obs_red);
    c->launches++;
    cn = nullptr;
    ws = c->obs_red;
    scale = 1.0;
  }
  k_obs_cols<<<g, kBlock, 0, c->stream>>>(cn, ws, c->cfg.nx, c->cfg.nk, na, c->dx, c->dk, scale,
                                          c->obs_density, c->obs_marg, c->obs_col);
  k_obs_total<<<1, kBlock, 0, c->stream>>>(c->obs_col, c->cfg.nx, c->cfg.xmin, c->dx, na,
                                           scale, c->obs_scalar);
  c->launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_transmissions(Ctx* c, const int* counts, double* out) {
  k_obs_trans<<<c->ninst, kBlock, 0, c->stream>>>(counts, c->cfg.nx, c->cfg.nk, c->cfg.xmin,
                                                  c->dx, c->inst_na, out);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_scan_tangent(Ctx* c) {
  const long long nb = c->scan_blocks;
  k_tcells_a<<<(unsigned)nb, kBlock, 0, c->stream>>>(c->dgrid[0], c->dgrid[1], c->nh, c->tquantum,
                                                    c->scan_bsum, c->scan_bnz);
  k_cells_b<<<1, kBlock, 0, c->stream>>>(c->scan_bsum, c->scan_bnz, nb, c->cnt, c->tile_cap,
                                         c->tinst_slot + c->ninst, 1);
  k_tcells_c<<<(unsigned)nb, kBlock, 0, c->stream>>>(c->dgrid[0], c->dgrid[1], c->nh, c->tquantum,
                                                    c->scan_bsum, c->scan_bnz, c->tnz_cell,
                                                    c->tnz_start, c->tnz_tau, c->ttile_nz,
                                                    c->tile_cap, c->nhi, c->tinst_slot);
  c->launches += 3;
  return cudaGetLastError();
}

cudaError_t launch_transmission_gradients(Ctx* c) {
  k_obs_tgrad<<<c->ninst, kBlock, 0, c->stream>>>(c->dgrid[0], c->dgrid[1], c->cfg.nx, c->cfg.nk,
                                                  c->cfg.xmin, c->dx, c->inst_na, c->inst_grad);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_live_instance(Ctx* c, int inst, unsigned long long* out) {
  k_live_inst<<<grid_cap(c, 4), kBlock, 0, c->stream>>>(c->cnt, c->inst_slot, c->cinst, inst, out);
  c->launches++;
  return cudaGetLastError();
}

}  // namespace wbrw

// ---------------------------------------------------------------------------
// Allocation-free observables (wbrw_observables_static in include/wbrw.h).
// For callers that cannot call cudaMalloc: the per-column scratch of the
// observables kernels is a file-scope device array of fixed size, looked up
// once per device with cudaGetSymbolAddress.  Host code must never pass the
// array's name itself to a kernel: on the host it names a stand-in, not the
// device copy.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {
constexpr int kStaticMaxDevices = 64;
static __device__ __align__(256) long long g_obs_col_static[WBRW_STATIC_MAX_NX];
std::mutex g_static_mu;
long long* g_static_col[kStaticMaxDevices];  // device address, per device

// A caller's buffer must be device (or managed) memory of the current
// device: the kernels below run there, and a buffer of another GPU or of the
// host would be read across the interconnect at best and fault at worst.
bool on_device(const void* ptr, int dev) {
  if (!ptr) return true;  // optional outputs
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();  // unregistered host memory: clear the query's error
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" wbrw_status wbrw_observables_static(const int* grid, int nx, int nk, double xmin,
                                               double xmax, double kmin, double kmax,
                                               long long n_alpha, double* density,
                                               double* marginal_x, double* transmission,
                                               void* cuda_stream) {
  if (!grid || !marginal_x || !transmission || nx <= 0 || nk <= 0 || n_alpha <= 0 ||
      !(xmax > xmin) || !(kmax > kmin) || (long long)nx * (long long)nk >= (1ll << 31))
    return WBRW_ERR_ARG;
  if (nx > WBRW_STATIC_MAX_NX) return WBRW_ERR_CAPACITY;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices)
    return WBRW_ERR_CUDA;
  if (!on_device(grid, dev) || !on_device(density, dev) || !on_device(marginal_x, dev) ||
      !on_device(transmission, dev))
    return WBRW_ERR_ARG;
  long long* col = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_col[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_obs_col_static) != cudaSuccess || !ptr)
        return WBRW_ERR_CUDA;
      g_static_col[dev] = (long long*)ptr;
    }
    col = g_static_col[dev];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const double na = (double)n_alpha;
  const double dx = (xmax - xmin) / (double)nx, dk = (kmax - kmin) / (double)nk;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return WBRW_ERR_CUDA;
  // Each launch is checked on its own.  cudaGetLastError also returns (and
  // clears) an error that an earlier runtime call of the caller left
  // pending; such an error is reported here as WBRW_ERR_CUDA.
  wbrw::k_obs_cols<<<4 * sms, wbrw::kBlock, 0, s>>>(grid, nullptr, nx, nk, na, dx, dk, 1.0, density,
                                                    marginal_x, col);
  if (cudaGetLastError() != cudaSuccess) return WBRW_ERR_CUDA;
  wbrw::k_obs_total<<<1, wbrw::kBlock, 0, s>>>(col, nx, xmin, dx, na, 1.0, transmission);
  if (cudaGetLastError() != cudaSuccess) return WBRW_ERR_CUDA;
  return WBRW_OK;
}
