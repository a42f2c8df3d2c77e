/*
 * wbrw_oracle.c -- plain FP64 CPU oracle of the signed-particle Wigner
 * branching random walk (Xiong & Shao, "The Wigner branching random walk:
 * efficient implementation and performance evaluation", arXiv:1709.02121).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library under paper_1709_02121_gb300/) never calls it, and the two
 * share no code, header, table or constant generator.
 *
 * It is written to be read against the paper, not to be fast:
 *   - one particle list in FP64, stepped one interval [t_l, t_{l+1}] at a time
 *     (Alg. 1), each particle processed on its own;
 *   - a recursion for the offspring born inside an interval (Alg. 1, item 3);
 *   - annihilation by the signed histogram (Eq. signed_histogram, Sec. 4.3)
 *     and regeneration by Alg. 3 without rounding (Remark after Alg. 3);
 *   - the signed residual bootstrap (Alg. 2 applied to S+ and S- separately,
 *     Eq. lambda / double_bootstrap / boostrap_histogram) followed by Alg. 3
 *     with stochastic rounding.
 *
 * Threads (optional, OpenMP): an interval's particle list is cut into as
 * many contiguous chunks as threads, each chunk's outputs go to its own list,
 * and the lists are joined in chunk order, so the result is the serial one
 * bit for bit; binning adds integers and regeneration writes each cell's
 * particles at their place in cell order.  The default is one thread.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11), implemented here from that
 * definition, keyed by the run seed and indexed by counters (particle id,
 * step, draw).  Every draw is named by its counter, so the order in which
 * particles are processed never changes a result.
 *
 * Pinned by tests/test_oracle_*.py against: an independent Philox
 * implementation, quadrature of the Wigner-kernel definition (Eq. 2), the
 * closed-form life-length (Sec. 3.2), exact free transport, conservation of
 * the net signed count, the growth bound of Theorem 1, the time-dependent
 * Schroedinger equation, a deterministic grid solver of the truncated Wigner
 * equation, and exact enumeration of the bootstrap law (Lemma 1 / Alg. 2).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TWO_PI 6.283185307179586476925286766559
#define ORC_PI 3.141592653589793238462643383280

/* Counter word 2 values reserved for streams that are not time steps. */
#define ORC_STEP_INIT 0xFFFFFFFFu  /* initial sampling from f0               */
#define ORC_STEP_REGEN 0xFFFFFFFEu /* in-cell offsets of Alg. 3              */
#define ORC_STEP_BOOT 0xFFFFFFFDu  /* residual draws of Alg. 2               */
#define ORC_STEP_ROUND 0xFFFFFFFCu /* rounding step of Alg. 3 (sp2 only)     */
#define ORC_DRAW_PIDS 0x80000000u  /* counter word 3 flag: offspring ids     */
#define ORC_DRAW_COMP 0x40000000u  /* counter word 3 flag: component choice  */
#define ORC_MAXC 4                 /* components of a time-dependent V       */

/* ------------------------------------------------------------------------ */
/* Philox4x32-10                                                             */
/* ------------------------------------------------------------------------ */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)prod1;
    uint32_t n2 = (uint32_t)(prod0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)prod0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* A double in [0,1) with 53 random bits: 27 from a, 26 from b. */
double orc_u53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) *
         (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------------ */
/* Gaussian barrier V(x) = H exp(-(x-xc)^2/(2w^2)) and its Wigner kernel      */
/* ------------------------------------------------------------------------ */

/* V_W(x,kappa) from the definition (Eq. 2) for a potential symmetric about
 * xc: V_W = (2/(pi hbar)) Vhat(2 kappa) sin(2 (x-xc) kappa), with
 * Vhat(q) = int V(z) exp(-i q z) dz.  For the Gaussian barrier
 * Vhat(q) = H w sqrt(2 pi) exp(-q^2 w^2 / 2).  (The prefactor printed in
 * Sec. 4.2 is half of this; the tests pin the derived one by quadrature of
 * the definition and by the rate printed in Sec. 5.5.) */
double orc_vw_gauss(double H, double w, double xc, double hbar, double x,
                    double kappa) {
  double vhat = H * w * sqrt(ORC_TWO_PI) * exp(-2.0 * kappa * kappa * w * w);
  return (2.0 / (ORC_PI * hbar)) * vhat * sin(2.0 * (x - xc) * kappa);
}

/* xi(x) = int V_W^+(x,kappa) dkappa (Eq. def.xi_m) for the Gaussian barrier.
 * With u = x - xc, V_W^+ integrates to (C/2) E|sin(theta)|, theta ~ N(0, s^2),
 * s = |u|/w, C = 2|H|/hbar.  From |sin t| = 2/pi - (4/pi) sum cos(2nt)/(4n^2-1)
 * and sum 1/(4n^2-1) = 1/2:
 *   E|sin theta| = (4/pi) sum_{n>=1} (1 - exp(-2 n^2 s^2)) / (4n^2-1),
 * summed to N with 2 N^2 s^2 >= 50 plus the exact tail sum_{n>N} 1/(4n^2-1)
 * = 1/(2(2N+1)).  For s < 1e-4 the two-term expansion
 * s sqrt(2/pi) (1 - s^2/3) of E|sin theta| is used instead. */
double orc_xi_gauss(double H, double w, double xc, double hbar, double x) {
  double s = fabs(x - xc) / w;
  double e;
  if (s < 1e-4) {
    e = s * sqrt(2.0 / ORC_PI) * (1.0 - s * s / 3.0);
  } else {
    double a = 2.0 * s * s;
    long long N = (long long)ceil(sqrt(50.0 / a)) + 1;
    double acc = 0.0;
    for (long long n = N; n >= 1; --n) /* small terms first */
      acc += -expm1(-a * (double)n * (double)n) /
             (4.0 * (double)n * (double)n - 1.0);
    acc += 1.0 / (2.0 * (2.0 * (double)N + 1.0));
    e = (4.0 / ORC_PI) * acc;
  }
  return (fabs(H) / hbar) * e;
}

/* ------------------------------------------------------------------------ */
/* Configuration and state                                                   */
/* ------------------------------------------------------------------------ */

/* One Gaussian component of a time-dependent potential (Remark 1):
 * V_m(x, t) = (a + b cos(om t + ph)) exp(-(x - xc)^2 / (2 w^2)). */
typedef struct {
  double a, b, om, ph, w, xc;
} orc_comp;

typedef struct {
  double hbar, mass, dt, gamma0; /* gamma0 <= 0 selects C/2                  */
  double H, w, xc;               /* Gaussian barrier                         */
  int nx, nk;                    /* histogram cells in x and k               */
  double xmin, xmax, kmin, kmax; /* histogram domain = truncation domain K   */
  int strategy;                  /* 1 = sp1 (pair generation), 2 = sp2,     */
                                 /* 3 = wp (weighted histogram)             */
  long long n_alpha;             /* sample size N_alpha of the estimator     */
  unsigned long long seed;
  int instance;                  /* id salt 0..255: a run as instance i of a batch */
  int tangent;                   /* sp1: carry the tangent weights (H, w)   */
  long long tquantum;            /* tangent particles: |tau| <= this / 2^32 */
  int ncomp;                     /* > 0: V is the sum of comp[0..ncomp), and */
  orc_comp comp[ORC_MAXC];       /* H, w, xc, gamma0 are not used           */
} orc_config;

typedef struct {
  double x, k, w; /* position, wavevector, signed weight (sp1: +-1, 0 for a  */
                  /* particle that only carries tangent weight)              */
  uint64_t pid;   /* counter-stream id                                       */
  double tH, tw;  /* tangent weights d/dH and d/dw (tangent mode)            */
} orc_particle;

typedef struct {
  uint64_t pid, pid_plus, pid_minus;
  uint32_t step, j;
  double t, xe, kappa, factor;
  int32_t kill_plus, kill_minus;
} orc_event;

enum {
  ORC_L_EVENTS = 0,  /* accepted events (pairs emitted)                 */
  ORC_L_KILL_P = 1,  /* + offspring killed outside K (Alg. 1, item 3)   */
  ORC_L_KILL_M = 2,  /* - offspring killed outside K                    */
  ORC_L_OUT_P = 3,   /* + particles outside the histogram at binning    */
  ORC_L_OUT_M = 4,   /* - particles outside the histogram at binning    */
  ORC_L_PSTEPS = 5,  /* sum over steps of particles alive at step start */
  ORC_L_CAND = 6,    /* candidate intervals: a particle alive at the start
                        of an interval has its first event inside it     */
  ORC_L_PAIRS0 = 7,  /* the candidate intervals whose first event emits  */
  ORC_L_N = 8
};

/* What the particles of one chunk produce in an interval: the next list,
 * ledger counts, the killed weights and the event log. */
typedef struct {
  orc_particle* q;
  long long nq, capq;
  long long ledger[ORC_L_N];
  double wkill[2], tkill[2];
  orc_event* log;
  long long nlog, logcap;
} orc_sink;

typedef struct {
  orc_config c;
  int threads;        /* chunks (and OpenMP threads) of an interval        */
  orc_sink* sink;     /* one per chunk                                     */
  double C, sig_k, gamma0, cacc, hm, dtv, dx, dk, inv_dx, inv_dk;
  double gam_c[ORC_MAXC];  /* component rates (time-dependent potential)      */
  uint32_t key[2];
  orc_particle* p;
  long long n, cap;
  int* grid;          /* signed int32 counts c_nu, nx*nk, x-major          */
  long long step;     /* index l of the next interval                      */
  long long epoch;    /* number of annihilations so far                    */
  int fresh;          /* 1 right after an annihilation                     */
  long long ledger[ORC_L_N];
  double wkill[2];    /* sp2: killed offspring weight, + and - sides       */
  orc_event* log;
  long long nlog, logcap;
  int log_on;
  /* sp2 diagnostics of the last filter */
  long long boot_n[2], boot_keep[2], boot_nr[2];
  unsigned long long boot_wfix[2];
  long long* boot_cnt[2]; /* n~_nu^+ and n~_nu^- of the last filter        */
  long long* dgrid[2];    /* tangent histogram D_nu (H, w) in units of 2^-32 */
  double tkill[2];        /* tangent weight of killed offspring, (H, w)      */
} orc_state;

static void draw4(const orc_state* s, uint64_t pid, uint32_t c2, uint32_t c3,
                  uint32_t out[4]) {
  uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)(pid >> 32), c2, c3};
  orc_philox4x32_10(ctr, s->key, out);
}

static int push(orc_particle** a, long long* n, long long* cap,
                orc_particle v) {
  if (*n == *cap) {
    long long nc = *cap ? *cap * 2 : 1024;
    orc_particle* b = (orc_particle*)realloc(*a, (size_t)nc * sizeof(**a));
    if (!b) return -1;
    *a = b;
    *cap = nc;
  }
  (*a)[(*n)++] = v;
  return 0;
}

orc_state* orc_create(const orc_config* c) {
  if (c->instance < 0 || c->instance >= 256 || c->nx <= 0 || c->nk <= 0 || !(c->xmax > c->xmin) ||
      !(c->kmax > c->kmin) || c->dt <= 0 || c->hbar <= 0 || c->mass <= 0 ||
      (c->strategy < 1 || c->strategy > 3) || c->n_alpha <= 0 || c->w <= 0)
    return NULL;
  if (c->tangent && (c->strategy != 1 || c->H == 0.0 || c->tquantum <= 0)) return NULL;
  if (c->ncomp < 0 || c->ncomp > ORC_MAXC || (c->ncomp > 0 && c->tangent)) return NULL;
  for (int m = 0; m < c->ncomp; ++m)
    if (!(c->comp[m].w > 0)) return NULL;
  orc_state* s = (orc_state*)calloc(1, sizeof(orc_state));
  s->c = *c;
  s->threads = 1;
  s->sink = (orc_sink*)calloc(1, sizeof(orc_sink));
  s->C = 2.0 * fabs(c->H) / c->hbar;          /* int |Vhat(2k)| (2/(pi hbar)) dk */
  s->sig_k = 1.0 / (2.0 * c->w);              /* proposal N(0, sig_k^2)          */
  s->gamma0 = c->gamma0 > 0 ? c->gamma0 : 0.5 * s->C;
  if (s->gamma0 <= 0) s->gamma0 = 1.0;        /* H = 0: any clock works          */
  s->cacc = s->C / (2.0 * s->gamma0);         /* xi_hat/gamma0 of Remark 3       */
  if (c->ncomp > 0) {
    /* Remark 1: a rate at or above every component's xi at every time; the
     * majorant C_m(t)/2 = |a + b cos(.)|/hbar <= (|a| + |b|)/hbar of each
     * component, summed for the clock. */
    double G = 0.0;
    for (int m = 0; m < c->ncomp; ++m) {
      s->gam_c[m] = (fabs(c->comp[m].a) + fabs(c->comp[m].b)) / c->hbar;
      G += s->gam_c[m];
    }
    s->gamma0 = G > 0.0 ? G : 1.0;
  }
  s->hm = c->hbar / c->mass;
  s->dtv = c->dt * s->hm;
  s->dx = (c->xmax - c->xmin) / (double)c->nx;
  s->dk = (c->kmax - c->kmin) / (double)c->nk;
  s->inv_dx = (double)c->nx / (c->xmax - c->xmin);
  s->inv_dk = (double)c->nk / (c->kmax - c->kmin);
  s->key[0] = (uint32_t)c->seed;
  s->key[1] = (uint32_t)(c->seed >> 32);
  s->grid = (int*)calloc((size_t)c->nx * (size_t)c->nk, sizeof(int));
  if (c->tangent)
    for (int d = 0; d < 2; ++d)
      s->dgrid[d] = (long long*)calloc((size_t)c->nx * (size_t)c->nk, sizeof(long long));
  return s;
}

static void free_sinks(orc_state* s) {
  for (int t = 0; t < s->threads; ++t) {
    free(s->sink[t].q);
    free(s->sink[t].log);
  }
  free(s->sink);
}

void orc_destroy(orc_state* s) {
  if (!s) return;
  free_sinks(s);
  free(s->p);
  free(s->grid);
  free(s->log);
  free(s->boot_cnt[0]);
  free(s->boot_cnt[1]);
  free(s->dgrid[0]);
  free(s->dgrid[1]);
  free(s);
}

int orc_cacc_ok(const orc_state* s) { return s->cacc <= 1.0; }
double orc_gamma0(const orc_state* s) { return s->gamma0; }

void orc_enable_log(orc_state* s, int on) { s->log_on = on; }

/* Threads the library was built for (1 without OpenMP). */
int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Cut each interval (and binning and regeneration) into n chunks, run by n
 * threads where OpenMP is available.  Results do not depend on n. */
int orc_set_threads(orc_state* s, int n) {
  if (n < 1) return -1;
  orc_sink* k = (orc_sink*)calloc((size_t)n, sizeof(orc_sink));
  if (!k) return -1;
  free_sinks(s);
  s->sink = k;
  s->threads = n;
  return 0;
}

int orc_threads(const orc_state* s) { return s->threads; }

/* ------------------------------------------------------------------------ */
/* Initial data: N particles from the Gaussian-wavepacket Wigner function     */
/* f0 = (1/pi) exp(-(x-x0)^2/(2 sx^2) - 2 sx^2 (k-k0)^2), which is positive:  */
/* x ~ N(x0, sx^2), k ~ N(k0, (1/(2 sx))^2), weight +1,                      */
/* pid = (instance << 32) | index.                                           */
/* ------------------------------------------------------------------------ */

int orc_init_gauss(orc_state* s, long long n, double x0, double sx,
                   double k0) {
  double sk = 1.0 / (2.0 * sx);
  s->n = 0;
  for (long long i = 0; i < n; ++i) {
    uint32_t r[4];
    const uint64_t pid0 = ((uint64_t)s->c.instance << 32) | (uint64_t)i;
    draw4(s, pid0, ORC_STEP_INIT, 0u, r);
    double ua = orc_u53(r[0], r[1]);
    double ub = orc_u53(r[2], r[3]);
    double rad = sqrt(-2.0 * log1p(-ua));
    double th = ORC_TWO_PI * ub;
    orc_particle p;
    p.x = x0 + sx * (rad * cos(th));
    p.k = k0 + sk * (rad * sin(th));
    p.w = 1.0;
    p.pid = pid0;
    p.tH = p.tw = 0.0;
    if (push(&s->p, &s->n, &s->cap, p)) return -1;
  }
  s->step = 0;
  s->epoch = 0;
  s->fresh = 0;
  return 0;
}

/* Load an explicit particle set (tests). */
int orc_set_particles(orc_state* s, long long n, const double* x,
                      const double* k, const double* w, const uint64_t* pid,
                      long long step) {
  s->n = 0;
  for (long long i = 0; i < n; ++i) {
    orc_particle p = {x[i], k[i], w[i], pid[i], 0.0, 0.0};
    if (push(&s->p, &s->n, &s->cap, p)) return -1;
  }
  s->step = step;
  s->fresh = 0;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Alg. 1 on one interval [t_l, t_{l+1}] for one particle segment.            */
/*                                                                          */
/* The segment starts at time to (0 for a particle present at t_l, the birth */
/* time for offspring) at position xo with wavevector k and weight w.        */
/* Life-lengths are exponential with the constant rate gamma0 and drawn     */
/* exactly, tau = -ln(1-u)/gamma0 (Sec. 3.2).  At each death the particle    */
/* is replaced by its copy (k' = k, w' = w) and, following the majorant     */
/* interpretation of Remark 3 with Vhat(2k) as proposal:                     */
/*   kappa ~ N(0, sig_k^2), i.e. the normalised |Vhat(2 kappa)|;             */
/*   sg = sin(2 (x - xc) kappa) is the ratio |V_W|/Vhat up to its sign;       */
/*   sp1: a pair is produced with probability cacc |sg| (rejection ratio),   */
/*        weights +w and -w;                                                 */
/*   sp2 (wp propagation): a pair is always produced with weights            */
/*        +w cacc |sg| and -w cacc |sg| (importance weight);                 */
/*   the pair is oriented by the sign of V_W(x, kappa) = sign(H) sign(sg)    */
/*   (Eq. 2: V_W carries the sign of Vhat, hence of H; the pair identity    */
/*   for 2 V_W/|V_W| in Sec. 3.1): + child at k + kappa', - child at        */
/*   k - kappa', kappa' = sign(H sg) kappa.                                 */
/* Offspring outside K are killed one by one (weight 0, Alg. 1 item 3).      */
/* Surviving offspring continue the same interval from their birth time.     */
/* ------------------------------------------------------------------------ */

/* Tangent mode (sp1, theta = (H, w)): each particle also carries a tangent
 * weight tau = s S, its sign s times the likelihood-ratio score S of its
 * lineage.  The expected particle measure is a sum over lineages of products
 * of the birth intensities V_W^+(x_b, kappa_b) (the parent survives every
 * birth, so no survival factor enters), hence the score of a lineage is the
 * sum over its births of g = d/dtheta log V_W^+(x_b, kappa_b; theta) =
 * (1/H, 1/w - 4 w kappa^2) for the Gaussian barrier (Eq. 2 with
 * Vhat(2 kappa) = H w sqrt(2 pi) exp(-2 w^2 kappa^2)).  A birth from (s, tau)
 * gives the + child (s, tau + s g) and the - child (-s, -(tau + s g)); the
 * parent keeps (s, tau).  Then d/dtheta E[sum_i s_i A(x_i, k_i)] =
 * E[sum_i tau_i A(x_i, k_i)] for any observable A. */
static int segment(const orc_state* s, orc_sink* o, double xo, double to, double k,
                   double w, uint64_t pid, uint32_t l, int is_root, double tH, double tw) {
  const orc_config* c = &s->c;
  uint32_t r[4];
  draw4(s, pid, l, 0u, r);
  double u0 = orc_u53(r[0], r[1]);
  double t = to + (-log1p(-u0) / s->gamma0);
  uint32_t j = 0;
  if (is_root && t < c->dt) o->ledger[ORC_L_CAND] += 1;
  while (t < c->dt) {
    double xe = xo + k * ((t - to) * s->hm);
    uint32_t a[4], b[4];
    draw4(s, pid, l, 1u + 2u * j, a);
    draw4(s, pid, l, 2u + 2u * j, b);
    double u1 = orc_u53(a[0], a[1]);
    double u2 = orc_u53(a[2], a[3]);
    double u3 = orc_u53(b[0], b[1]);
    double u4 = orc_u53(b[2], b[3]);
    double z = sqrt(-2.0 * log1p(-u1)) * cos(ORC_TWO_PI * u2);
    double kap, sg, f;
    int flip;
    if (c->ncomp == 0) {
      kap = s->sig_k * z;
      sg = sin(2.0 * (xe - c->xc) * kap);
      f = s->cacc * fabs(sg);
      flip = c->H < 0.0 ? sg > 0.0 : sg < 0.0;
    } else {
      /* time-dependent V (Remark 1): component m with probability
       * gamma_m/gamma0 (uniform uc of the draw (pid, l, COMP | j)), its
       * height H_m(t) at the absolute time t_l + t of the event, the kick
       * N(0, (1/(2 w_m))^2) and the acceptance |H_m(t)|/(hbar gamma_m)
       * |sin(2 (xe - xc_m) kappa)| (the component's majorant ratio) */
      uint32_t cc[4];
      draw4(s, pid, l, ORC_DRAW_COMP | j, cc);
      double v = orc_u53(cc[0], cc[1]) * s->gamma0;
      int m = 0;
      double acc = s->gam_c[0];
      while (m + 1 < c->ncomp && !(v < acc)) acc += s->gam_c[++m];
      const orc_comp* q = &c->comp[m];
      double ta = (double)l * c->dt + t;
      double Hm = q->a + q->b * cos(q->om * ta + q->ph);
      kap = (1.0 / (2.0 * q->w)) * z;
      sg = sin(2.0 * (xe - q->xc) * kap);
      f = s->gam_c[m] > 0.0 ? fabs(Hm) / (c->hbar * s->gam_c[m]) * fabs(sg) : 0.0;
      flip = Hm < 0.0 ? sg > 0.0 : sg < 0.0;
    }
    int emit;
    double wc;
    if (c->strategy == 1) {
      emit = u3 < f;
      wc = w;
    } else {
      emit = f > 0.0;
      wc = w * f;
    }
    if (emit) {
      if (flip) kap = -kap;
      uint32_t h[4];
      draw4(s, pid, l, ORC_DRAW_PIDS | j, h);
      uint64_t pid_p =
          (1ull << 63) | ((((uint64_t)h[1] << 32) | (uint64_t)h[0]) >> 1);
      uint64_t pid_m =
          (1ull << 63) | ((((uint64_t)h[3] << 32) | (uint64_t)h[2]) >> 1);
      double kp = k + kap, km = k - kap;
      int kill_p = !(kp >= c->kmin && kp < c->kmax);
      int kill_m = !(km >= c->kmin && km < c->kmax);
      o->ledger[ORC_L_EVENTS] += 1;
      if (is_root && j == 0) o->ledger[ORC_L_PAIRS0] += 1;
      double wp = wc, wm = -wc; /* + child carries +wc, - child -wc */
      double gH = 1.0 / c->H, gw = 1.0 / c->w - 4.0 * c->w * kap * kap;
      double tpH = tH + w * gH, tpw = tw + w * gw; /* + child's tangent    */
      if (kill_p) {
        if (wp > 0) o->ledger[ORC_L_KILL_P] += 1; else if (wp < 0) o->ledger[ORC_L_KILL_M] += 1;
        if (wp > 0) o->wkill[0] += wp; else o->wkill[1] += -wp;
      }
      if (kill_m) {
        if (wm > 0) o->ledger[ORC_L_KILL_P] += 1; else if (wm < 0) o->ledger[ORC_L_KILL_M] += 1;
        if (wm > 0) o->wkill[0] += wm; else o->wkill[1] += -wm;
      }
      if (c->tangent) {
        if (kill_p) { o->tkill[0] += tpH; o->tkill[1] += tpw; }
        if (kill_m) { o->tkill[0] -= tpH; o->tkill[1] -= tpw; }
      }
      if (s->log_on) {
        if (o->nlog == o->logcap) {
          long long nc = o->logcap ? o->logcap * 2 : 1024;
          orc_event* b2 = (orc_event*)realloc(o->log, (size_t)nc * sizeof(orc_event));
          if (!b2) return -1;
          o->log = b2;
          o->logcap = nc;
        }
        orc_event e;
        e.pid = pid;
        e.pid_plus = pid_p;
        e.pid_minus = pid_m;
        e.step = l;
        e.j = j;
        e.t = t;
        e.xe = xe;
        e.kappa = kap;
        e.factor = f;
        e.kill_plus = kill_p;
        e.kill_minus = kill_m;
        o->log[o->nlog++] = e;
      }
      if (!kill_p && segment(s, o, xe, t, kp, wp, pid_p, l, 0, tpH, tpw)) return -1;
      if (!kill_m && segment(s, o, xe, t, km, wm, pid_m, l, 0, -tpH, -tpw)) return -1;
    }
    t += -log1p(-u4) / s->gamma0;
    ++j;
  }
  orc_particle out;
  out.x = is_root ? xo + k * s->dtv : xo + k * ((c->dt - to) * s->hm);
  out.k = k;
  out.w = w;
  out.pid = pid;
  out.tH = tH;
  out.tw = tw;
  return push(&o->q, &o->nq, &o->capq, out);
}

/* Advance nsteps intervals (Alg. 1 applied interval by interval).  Chunk t
 * of the particle list is [t n / T, (t + 1) n / T); the chunks' next lists,
 * joined in chunk order, are the next list of a serial pass. */
static int join_sinks(orc_state* s) {
  const int T = s->threads;
  long long total = 0;
  for (int t = 0; t < T; ++t) total += s->sink[t].nq;
  if (T == 1) {  /* the chunk's list becomes the particle list */
    orc_sink* o = &s->sink[0];
    orc_particle* tp = s->p;
    long long tc = s->cap;
    s->p = o->q;
    s->cap = o->capq;
    o->q = tp;
    o->capq = tc;
  } else {
    if (total > s->cap) {
      orc_particle* b = (orc_particle*)realloc(s->p, (size_t)total * sizeof(orc_particle));
      if (!b) return -1;
      s->p = b;
      s->cap = total;
    }
    long long off[T + 1];
    off[0] = 0;
    for (int t = 0; t < T; ++t) off[t + 1] = off[t] + s->sink[t].nq;
#pragma omp parallel for num_threads(T) schedule(static, 1)
    for (int t = 0; t < T; ++t)
      if (s->sink[t].nq)
        memcpy(s->p + off[t], s->sink[t].q, (size_t)s->sink[t].nq * sizeof(orc_particle));
  }
  s->n = total;
  for (int t = 0; t < T; ++t) {
    orc_sink* o = &s->sink[t];
    for (int i = 0; i < ORC_L_N; ++i) s->ledger[i] += o->ledger[i];
    for (int d = 0; d < 2; ++d) {
      s->wkill[d] += o->wkill[d];
      s->tkill[d] += o->tkill[d];
    }
    if (o->nlog) {
      if (s->nlog + o->nlog > s->logcap) {
        long long nc = s->nlog + o->nlog + 1024;
        orc_event* b2 = (orc_event*)realloc(s->log, (size_t)nc * sizeof(orc_event));
        if (!b2) return -1;
        s->log = b2;
        s->logcap = nc;
      }
      memcpy(s->log + s->nlog, o->log, (size_t)o->nlog * sizeof(orc_event));
      s->nlog += o->nlog;
    }
  }
  return 0;
}

int orc_step(orc_state* s, int nsteps) {
  const int T = s->threads;
  for (int it = 0; it < nsteps; ++it) {
    uint32_t l = (uint32_t)s->step;
    s->ledger[ORC_L_PSTEPS] += s->n;
    int fail = 0;
#pragma omp parallel for num_threads(T) schedule(static, 1) reduction(| : fail)
    for (int t = 0; t < T; ++t) {
      orc_sink* o = &s->sink[t];
      o->nq = 0;
      o->nlog = 0;
      memset(o->ledger, 0, sizeof(o->ledger));
      o->wkill[0] = o->wkill[1] = o->tkill[0] = o->tkill[1] = 0.0;
      const long long i0 = s->n * t / T, i1 = s->n * (t + 1) / T;
      for (long long i = i0; i < i1 && !fail; ++i) {
        const orc_particle p = s->p[i];
        if (segment(s, o, p.x, 0.0, p.k, p.w, p.pid, l, 1, p.tH, p.tw)) fail = 1;
      }
    }
    if (fail || join_sinks(s)) return -1;
    s->step += 1;
    s->fresh = 0;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Histogram cells D_nu = X_ix x K_ik on the uniform mesh (Sec. 4.3).         */
/* ------------------------------------------------------------------------ */

static int cell_of(const orc_state* s, double x, double k, long long* nu) {
  double fx = floor((x - s->c.xmin) * s->inv_dx);
  double fk = floor((k - s->c.kmin) * s->inv_dk);
  if (!(fx >= 0.0 && fx < (double)s->c.nx && fk >= 0.0 &&
        fk < (double)s->c.nk))
    return 0;
  *nu = (long long)fx * s->c.nk + (long long)fk;
  return 1;
}

static double bin_x(const orc_state* s, double x) {
  return floor((x - s->c.xmin) * s->inv_dx);
}
static double bin_k(const orc_state* s, double k) {
  return floor((k - s->c.kmin) * s->inv_dk);
}

/* Alg. 3 for the signed counts c_nu already in s->grid: |c_nu| particles of
 * sign sign(c_nu), uniform in D_nu.  Particle j of the new list (cells in
 * order) gets pid = (epoch << 40) | (instance << 32) | j and its two
 * offsets from its own stream.  A coordinate that rounds onto a neighbouring cell is moved by
 * single ulps back into D_nu, so that binning the regenerated set gives the
 * same counts. */
/* One regenerated particle of cell (ix, ik): offsets from its own stream. */
static orc_particle regen_one(const orc_state* s, uint64_t pid, long long ix, long long ik,
                              double w, double tH, double tw) {
  uint32_t h[4];
  draw4(s, pid, ORC_STEP_REGEN, 0u, h);
  double x = s->c.xmin + ((double)ix + orc_u53(h[0], h[1])) * s->dx;
  double k = s->c.kmin + ((double)ik + orc_u53(h[2], h[3])) * s->dk;
  while (bin_x(s, x) > (double)ix) x = nextafter(x, -INFINITY);
  while (bin_x(s, x) < (double)ix) x = nextafter(x, INFINITY);
  while (bin_k(s, k) > (double)ik) k = nextafter(k, -INFINITY);
  while (bin_k(s, k) < (double)ik) k = nextafter(k, INFINITY);
  orc_particle p = {x, k, w, pid, tH, tw};
  return p;
}

static int regenerate(orc_state* s) {
  const long long nh = (long long)s->c.nx * s->c.nk;
  const int T = s->threads;
  /* chunk t holds cells [t nh / T, (t + 1) nh / T); its particles start
   * after those of the chunks before it */
  long long off[T + 1];
  off[0] = 0;
  for (int t = 0; t < T; ++t) {
    long long m = 0;
    for (long long nu = nh * t / T; nu < nh * (t + 1) / T; ++nu) m += llabs((long long)s->grid[nu]);
    off[t + 1] = off[t] + m;
  }
  if (off[T] > s->cap) {
    orc_particle* b = (orc_particle*)realloc(s->p, (size_t)off[T] * sizeof(orc_particle));
    if (!b) return -1;
    s->p = b;
    s->cap = off[T];
  }
#pragma omp parallel for num_threads(T) schedule(static, 1)
  for (int t = 0; t < T; ++t) {
    uint64_t j = (uint64_t)off[t];
    for (long long nu = nh * t / T; nu < nh * (t + 1) / T; ++nu) {
      int cnt = s->grid[nu];
      if (cnt == 0) continue;
      long long ix = nu / s->c.nk, ik = nu % s->c.nk;
      long long m = cnt > 0 ? cnt : -(long long)cnt;
      double sign = cnt > 0 ? 1.0 : -1.0;
      for (long long r = 0; r < m; ++r, ++j) {
        uint64_t pid = ((uint64_t)s->epoch << 40) | ((uint64_t)s->c.instance << 32) | j;
        s->p[j] = regen_one(s, pid, ix, ik, sign, 0.0, 0.0);
      }
    }
  }
  s->n = off[T];
  if (!s->c.tangent) return 0;
  /* Tangent mode: the tangent histogram D_nu is carried by particles of
   * sign 0, n_t = ceil(max(|D_H|, |D_w|) / quantum) of them per cell with
   * tau = D_nu / n_t each, uniform in D_nu (Alg. 3's offsets); their ids
   * are (epoch << 40) | (instance << 32) | 2^31 | j, j counting them in cell
   * order.  The signed particles carry tau = 0. */
  uint64_t jt = 0;
  for (long long nu = 0; nu < nh; ++nu) {
    long long dH = s->dgrid[0][nu], dw = s->dgrid[1][nu];
    long long m = llabs(dH) > llabs(dw) ? llabs(dH) : llabs(dw);
    if (m == 0) continue;
    long long nt = (m + s->c.tquantum - 1) / s->c.tquantum;
    long long ix = nu / s->c.nk, ik = nu % s->c.nk;
    double tH = (double)dH * (1.0 / 4294967296.0) / (double)nt;
    double tw = (double)dw * (1.0 / 4294967296.0) / (double)nt;
    for (long long r = 0; r < nt; ++r, ++jt) {
      uint64_t pid = ((uint64_t)s->epoch << 40) | ((uint64_t)s->c.instance << 32) |
                     0x80000000ull | jt;
      if (push(&s->p, &s->n, &s->cap, regen_one(s, pid, ix, ik, 0.0, tH, tw))) return -1;
    }
  }
  return 0;
}

/* sp1: signed histogram c_nu = n_nu^+ - n_nu^- (Eq. signed_histogram). */
/* In tangent mode also D_nu = sum of tau over the particles in D_nu, each
 * tau rounded to a multiple of 2^-32 (so the sum is exact and independent
 * of order); sign-0 particles enter D only. */
static void bin_signed(orc_state* s) {
  long long nh = (long long)s->c.nx * s->c.nk;
  memset(s->grid, 0, (size_t)nh * sizeof(int));
  if (s->c.tangent)
    for (int d = 0; d < 2; ++d) memset(s->dgrid[d], 0, (size_t)nh * sizeof(long long));
  long long out_p = 0, out_m = 0;
  /* integer sums: the same in any order */
#pragma omp parallel for num_threads(s->threads) reduction(+ : out_p, out_m)
  for (long long i = 0; i < s->n; ++i) {
    long long nu;
    const orc_particle* p = &s->p[i];
    if (cell_of(s, p->x, p->k, &nu)) {
      if (p->w != 0.0) {
#pragma omp atomic
        s->grid[nu] += p->w > 0 ? 1 : -1;
      }
      if (s->c.tangent) {
        const long long a = llrint(p->tH * 4294967296.0), b = llrint(p->tw * 4294967296.0);
#pragma omp atomic
        s->dgrid[0][nu] += a;
#pragma omp atomic
        s->dgrid[1][nu] += b;
      }
    } else {
      if (p->w > 0) out_p += 1; else if (p->w < 0) out_m += 1;
    }
  }
  s->ledger[ORC_L_OUT_P] += out_p;
  s->ledger[ORC_L_OUT_M] += out_m;
}

static uint64_t mulhi64(uint64_t a, uint64_t b) {
  return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
}

/* sp2: the signed residual bootstrap (Alg. 2 on S+ and S-, Eq. lambda,
 * Eq. double_bootstrap) followed by the histogram of Eq. boostrap_histogram
 * and the rounding step of Alg. 3.
 *
 * Fixed-point conventions (so that the sums are exact and order-free):
 *   |w_i| -> a_i = floor(|w_i| 2^31)             (Q1.31, a_i <= 2^31)
 *   W^s  = sum_{i in S^s} a_i                    (uint64; W^s 2^-31 = sum |w|)
 *   q_i  = a_i * (N^s / W^s)                     (FP64; sum_i q_i = N^s)
 *   keep_i = floor(q_i); res_i = floor((q_i - keep_i) 2^32)  (Q0.32)
 *   N_r^s = N^s - sum keep_i draws, each picking cell nu with probability
 *   R_nu / R (R_nu = residual sum of the side in nu): only the cell of a
 *   draw enters the histogram, so this has the law of drawing particles.
 * Draw d of side s: r = 64 random bits, U = floor(r R / 2^64), cell = the
 * first nu whose inclusive prefix of R exceeds U.  The draw's counter is
 * (instance << 32) | d and the rounding of cell nu's is (instance << 32) | nu,
 * so that the instances of a batch (salt 0 for a plain run) draw from
 * separate streams, as their particle labels do.
 * Then m_nu = (W^+/N^+) n~_nu^+ - (W^-/N^-) n~_nu^-  (= N_alpha mu(D_nu)
 * d_nu of Alg. 3) and |m_nu| is rounded stochastically with its own u. */
static int bootstrap(orc_state* s) {
  long long nh = (long long)s->c.nx * s->c.nk;
  long long* cell = (long long*)malloc((size_t)(s->n ? s->n : 1) * sizeof(long long));
  int* side = (int*)malloc((size_t)(s->n ? s->n : 1) * sizeof(int));
  uint32_t* a = (uint32_t*)malloc((size_t)(s->n ? s->n : 1) * sizeof(uint32_t));
  long long* keep[2];
  uint64_t* res[2];
  for (int sd = 0; sd < 2; ++sd) {
    keep[sd] = (long long*)calloc((size_t)nh, sizeof(long long));
    res[sd] = (uint64_t*)calloc((size_t)nh, sizeof(uint64_t));
  }
  long long N[2] = {0, 0};
  uint64_t W[2] = {0, 0};
  for (long long i = 0; i < s->n; ++i) {
    double w = s->p[i].w;
    long long nu;
    side[i] = -1;
    if (!cell_of(s, s->p[i].x, s->p[i].k, &nu)) {
      if (w > 0) s->ledger[ORC_L_OUT_P] += 1; else if (w < 0) s->ledger[ORC_L_OUT_M] += 1;
      continue;
    }
    if (w == 0.0) continue;
    int sd = w > 0 ? 0 : 1;
    side[i] = sd;
    cell[i] = nu;
    a[i] = (uint32_t)floor(fabs(w) * 2147483648.0);
    N[sd] += 1;
    W[sd] += a[i];
  }
  double ratio[2];
  for (int sd = 0; sd < 2; ++sd)
    ratio[sd] = W[sd] > 0 ? (double)N[sd] / (double)W[sd] : 0.0;
  long long ksum[2] = {0, 0};
  for (long long i = 0; i < s->n; ++i) {
    int sd = side[i];
    if (sd < 0) continue;
    double q = (double)a[i] * ratio[sd];
    double fl = floor(q);
    keep[sd][cell[i]] += (long long)fl;
    ksum[sd] += (long long)fl;
    res[sd][cell[i]] += (uint64_t)floor((q - fl) * 4294967296.0);
  }
  for (int sd = 0; sd < 2; ++sd) {
    long long nr = N[sd] - ksum[sd];
    if (nr < 0) nr = 0;
    s->boot_n[sd] = N[sd];
    s->boot_keep[sd] = ksum[sd];
    s->boot_nr[sd] = nr;
    s->boot_wfix[sd] = W[sd];
    uint64_t* pre = (uint64_t*)malloc((size_t)nh * sizeof(uint64_t));
    uint64_t acc = 0;
    for (long long nu = 0; nu < nh; ++nu) {
      acc += res[sd][nu];
      pre[nu] = acc;
    }
    uint64_t R = acc;
    if (R > 0) {
      for (long long d = 0; d < nr; ++d) {
        uint32_t h[4];
        draw4(s, ((uint64_t)s->c.instance << 32) | (uint64_t)d, ORC_STEP_BOOT,
              (uint32_t)(((uint64_t)s->epoch << 1) | (uint64_t)sd), h);
        uint64_t r64 = ((uint64_t)h[1] << 32) | (uint64_t)h[0];
        uint64_t U = mulhi64(r64, R);
        long long lo = 0, hi = nh - 1; /* first nu with pre[nu] > U */
        while (lo < hi) {
          long long mid = lo + (hi - lo) / 2;
          if (pre[mid] > U) hi = mid; else lo = mid + 1;
        }
        keep[sd][lo] += 1;
      }
    }
    free(pre);
  }
  double amp[2];
  for (int sd = 0; sd < 2; ++sd)
    amp[sd] = N[sd] > 0 ? ((double)W[sd] * (1.0 / 2147483648.0)) / (double)N[sd] : 0.0;
  for (int sd = 0; sd < 2; ++sd) {
    if (!s->boot_cnt[sd]) s->boot_cnt[sd] = (long long*)malloc((size_t)nh * sizeof(long long));
    memcpy(s->boot_cnt[sd], keep[sd], (size_t)nh * sizeof(long long));
  }
  for (long long nu = 0; nu < nh; ++nu) {
    double m = (double)keep[0][nu] * amp[0] - (double)keep[1][nu] * amp[1];
    double am = fabs(m);
    double fl = floor(am);
    uint32_t h[4];
    draw4(s, ((uint64_t)s->c.instance << 32) | (uint64_t)nu, ORC_STEP_ROUND,
          (uint32_t)s->epoch, h);
    double u = orc_u53(h[0], h[1]);
    long long cnt = (long long)fl + (u < am - fl ? 1 : 0);
    s->grid[nu] = (int)(m < 0 ? -cnt : cnt);
  }
  for (int sd = 0; sd < 2; ++sd) {
    free(keep[sd]);
    free(res[sd]);
  }
  free(cell);
  free(side);
  free(a);
  return 0;
}

/* Resampling (Sec. 4.3): histogram, then Alg. 3.  A second call with no step
 * in between changes nothing. */
/* wp: the weighted histogram of Eq. piecewise_constant_function, sum_i w_i
 * over D_nu (each w in fixed point, llrint(w 2^31), so the sum is exact),
 * then Alg. 3 with its rounding step: floor(|m|) particles plus one with
 * probability |m| - floor(|m|), of sign sign(m), from the uniform of the
 * draw ((instance << 32) | nu, ROUND, epoch) as for sp2. */
static int wp_histogram(orc_state* s) {
  long long nh = (long long)s->c.nx * s->c.nk;
  long long* ws = (long long*)calloc((size_t)nh, sizeof(long long));
  if (!ws) return -1;
  for (long long i = 0; i < s->n; ++i) {
    long long nu;
    const orc_particle* p = &s->p[i];
    if (cell_of(s, p->x, p->k, &nu)) {
      ws[nu] += llrint(p->w * 2147483648.0);
    } else {
      if (p->w > 0) s->ledger[ORC_L_OUT_P] += 1; else if (p->w < 0) s->ledger[ORC_L_OUT_M] += 1;
    }
  }
  for (long long nu = 0; nu < nh; ++nu) {
    double m = (double)ws[nu] * (1.0 / 2147483648.0);
    double am = fabs(m);
    double fl = floor(am);
    uint32_t h[4];
    draw4(s, ((uint64_t)s->c.instance << 32) | (uint64_t)nu, ORC_STEP_ROUND,
          (uint32_t)s->epoch, h);
    double u = orc_u53(h[0], h[1]);
    long long cnt = (long long)fl + (u < am - fl ? 1 : 0);
    s->grid[nu] = (int)(m < 0 ? -cnt : cnt);
  }
  free(ws);
  return 0;
}

int orc_annihilate(orc_state* s) {
  if (s->fresh) return 0;
  s->epoch += 1;
  if (s->c.strategy == 1) {
    bin_signed(s);
  } else if (s->c.strategy == 3) {
    if (wp_histogram(s)) return -1;
  } else {
    if (bootstrap(s)) return -1;
  }
  if (regenerate(s)) return -1;
  s->fresh = 1;
  return 0;
}

/* Histogram of the current particles without resampling: sp1 signed counts
 * into counts (int), and the signed weights (FP64) into wsum for both. */
void orc_histogram(const orc_state* s, int* counts, double* wsum) {
  long long nh = (long long)s->c.nx * s->c.nk;
  if (counts) memset(counts, 0, (size_t)nh * sizeof(int));
  if (wsum) memset(wsum, 0, (size_t)nh * sizeof(double));
  for (long long i = 0; i < s->n; ++i) {
    long long nu;
    if (!cell_of(s, s->p[i].x, s->p[i].k, &nu)) continue;
    if (counts) counts[nu] += s->p[i].w > 0 ? 1 : (s->p[i].w < 0 ? -1 : 0);
    if (wsum) wsum[nu] += s->p[i].w;
  }
}

/* Observables (Eq. estimator with A = indicator of a cell, of an x-column,
 * of x > 0): density c_nu/(N_alpha mu(D_nu)), x-marginal and transmission
 * from signed counts. */
void orc_observables(const orc_state* s, const int* counts, double* density,
                     double* marginal_x, double* transmission) {
  const orc_config* c = &s->c;
  double na = (double)c->n_alpha;
  double T = 0.0;
  for (int ix = 0; ix < c->nx; ++ix) {
    long long col = 0;
    for (int ik = 0; ik < c->nk; ++ik) {
      long long nu = (long long)ix * c->nk + ik;
      col += counts[nu];
      if (density) density[nu] = (double)counts[nu] / (na * s->dx * s->dk);
    }
    if (marginal_x) marginal_x[ix] = (double)col / (na * s->dx);
    double centre = c->xmin + ((double)ix + 0.5) * s->dx;
    if (centre > 0.0) T += (double)col;
  }
  if (transmission) *transmission = T / na;
}

/* ------------------------------------------------------------------------ */
/* Accessors                                                                 */
/* ------------------------------------------------------------------------ */

long long orc_count(const orc_state* s) { return s->n; }
long long orc_step_index(const orc_state* s) { return s->step; }
long long orc_epoch(const orc_state* s) { return s->epoch; }

void orc_get_particles(const orc_state* s, double* x, double* k, double* w,
                       uint64_t* pid) {
  for (long long i = 0; i < s->n; ++i) {
    if (x) x[i] = s->p[i].x;
    if (k) k[i] = s->p[i].k;
    if (w) w[i] = s->p[i].w;
    if (pid) pid[i] = s->p[i].pid;
  }
}

void orc_get_grid(const orc_state* s, int* grid) {
  memcpy(grid, s->grid, (size_t)s->c.nx * (size_t)s->c.nk * sizeof(int));
}

void orc_set_grid(orc_state* s, const int* grid, long long epoch) {
  memcpy(s->grid, grid, (size_t)s->c.nx * (size_t)s->c.nk * sizeof(int));
  s->epoch = epoch;
}

int orc_regenerate(orc_state* s) {
  s->fresh = 1;
  return regenerate(s);
}

void orc_get_ledger(const orc_state* s, long long* out) {
  for (int i = 0; i < ORC_L_N; ++i) out[i] = s->ledger[i];
}

void orc_get_tangent(const orc_state* s, double* tH, double* tw) {
  for (long long i = 0; i < s->n; ++i) {
    if (tH) tH[i] = s->p[i].tH;
    if (tw) tw[i] = s->p[i].tw;
  }
}

void orc_get_dgrid(const orc_state* s, long long* dH, long long* dw) {
  size_t nh = (size_t)s->c.nx * (size_t)s->c.nk;
  if (dH && s->dgrid[0]) memcpy(dH, s->dgrid[0], nh * sizeof(long long));
  if (dw && s->dgrid[1]) memcpy(dw, s->dgrid[1], nh * sizeof(long long));
}

void orc_get_tkill(const orc_state* s, double* out) {
  out[0] = s->tkill[0];
  out[1] = s->tkill[1];
}

/* d/dtheta of the transmission estimate from the tangent histogram: the sum
 * of D_nu over cells with centre x > 0, divided by N_alpha. */
void orc_tangent_transmission(const orc_state* s, double* out) {
  const orc_config* c = &s->c;
  long long acc[2] = {0, 0};
  for (int ix = 0; ix < c->nx; ++ix) {
    double centre = c->xmin + ((double)ix + 0.5) * s->dx;
    if (!(centre > 0.0)) continue;
    for (int ik = 0; ik < c->nk; ++ik)
      for (int d = 0; d < 2; ++d) acc[d] += s->dgrid[d][(long long)ix * c->nk + ik];
  }
  for (int d = 0; d < 2; ++d)
    out[d] = (double)acc[d] * (1.0 / 4294967296.0) / (double)c->n_alpha;
}

void orc_get_wkill(const orc_state* s, double* out) {
  out[0] = s->wkill[0];
  out[1] = s->wkill[1];
}

void orc_get_boot(const orc_state* s, long long* n, long long* keep,
                  long long* nr, unsigned long long* wfix) {
  for (int sd = 0; sd < 2; ++sd) {
    n[sd] = s->boot_n[sd];
    keep[sd] = s->boot_keep[sd];
    nr[sd] = s->boot_nr[sd];
    wfix[sd] = s->boot_wfix[sd];
  }
}

/* n~_nu^+ and n~_nu^- of the last sp2 filter (zeros before the first). */
void orc_get_boot_counts(const orc_state* s, long long* plus, long long* minus) {
  long long nh = (long long)s->c.nx * s->c.nk;
  for (long long nu = 0; nu < nh; ++nu) {
    plus[nu] = s->boot_cnt[0] ? s->boot_cnt[0][nu] : 0;
    minus[nu] = s->boot_cnt[1] ? s->boot_cnt[1][nu] : 0;
  }
}

long long orc_log_count(const orc_state* s) { return s->nlog; }

void orc_get_log(const orc_state* s, orc_event* out) {
  memcpy(out, s->log, (size_t)s->nlog * sizeof(orc_event));
}

long long orc_event_size(void) { return (long long)sizeof(orc_event); }

/* The event outcome alone, for sampler tests: the candidate event j of
 * particle pid in interval l at position xe, as segment() decides it.
 * Returns 1 if a pair is emitted; *kappa gets the oriented kick, *factor the
 * acceptance ratio / weight factor cacc |sg|, *gap the next exponential gap. */
int orc_event_outcome(const orc_state* s, uint64_t pid, uint32_t l, uint32_t j,
                      double xe, double* kappa, double* factor, double* gap) {
  uint32_t a[4], b[4];
  draw4(s, pid, l, 1u + 2u * j, a);
  draw4(s, pid, l, 2u + 2u * j, b);
  double u1 = orc_u53(a[0], a[1]);
  double u2 = orc_u53(a[2], a[3]);
  double u3 = orc_u53(b[0], b[1]);
  double u4 = orc_u53(b[2], b[3]);
  double z = sqrt(-2.0 * log1p(-u1)) * cos(ORC_TWO_PI * u2);
  double kap = s->sig_k * z;
  double sg = sin(2.0 * (xe - s->c.xc) * kap);
  double f = s->cacc * fabs(sg);
  int emit = s->c.strategy == 1 ? (u3 < f) : (f > 0.0);
  if (s->c.H < 0.0 ? sg > 0.0 : sg < 0.0) kap = -kap;
  *kappa = kap;
  *factor = f;
  *gap = -log1p(-u4) / s->gamma0;
  return emit;
}
