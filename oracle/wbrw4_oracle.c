/*
 * wbrw4_oracle.c -- plain FP64 CPU oracle of the signed-particle WBRW for the
 * 4D Helium-like system of Example 1 (Xiong & Shao, arXiv:1709.02121): two
 * 1D electrons (x1, x2, k1, k2) in the field of a nucleus at xc,
 *   V = -Z/sqrt((x1-xc)^2 + a^2) - Z/sqrt((x2-xc)^2 + a^2)
 *       + lam/sqrt((x1-x2)^2 + a^2)
 * (soft-Coulomb terms in place of the paper's Yukawa ones).
 *
 * TEST INFRASTRUCTURE ONLY, like wbrw_oracle.c (whose Philox4x32-10 it uses):
 * the product library never calls it and shares no code with it.
 *
 * The method, written out in the paper's order:
 *   - the Wigner kernel splits into M = 3 components (Eq. M): the one-body
 *     terms act on k1 (argument y = x1 - xc) and on k2 (y = x2 - xc); the
 *     interaction, through the Fourier completeness relation of Example 1,
 *     is a 1D kernel in y = x1 - x2 that kicks k1 by +kappa and k2 by
 *     -kappa (the integral I_3 of Example 1).  From Eq. 2 each component is
 *       V_W,m(y, kappa) = (2/(pi hbar)) q_m Uhat(2 kappa) sin(2 y kappa),
 *     with Uhat(q) = 2 K0(a |q|) the transform of 1/sqrt(y^2 + a^2), and
 *     charges q = -Z (one-body) and lam (interaction);
 *   - V_W,m^+(y, .) is tabulated on a mesh of y nodes x kappa cells, with
 *     xi_m on the y nodes and linear interpolation between nodes, as Sec. 4.2
 *     advises for xi (Eq. def.xi_m);
 *   - the life-lengths of Alg. 1 are exponential with the constant rate
 *     Gamma = sum_m gamma_m, gamma_m >= max xi_m (Sec. 3.2); a death picks
 *     component m with probability gamma_m/Gamma and creates a +/- pair with
 *     probability xi_m(y)/gamma_m, the kick kappa drawn from
 *     V_W,m^+(y, .)/xi_m(y) by inverse CDF on the table row (a stand-in for
 *     the rejection sampler of Alg. 4);
 *   - annihilation (Eq. signed_histogram) and Alg. 3 on the 4D uniform mesh.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O4_PI 3.141592653589793238462643383280
#define O4_TWO_PI 6.283185307179586476925286766559

#define O4_STEP_INIT 0xFFFFFFFFu
#define O4_STEP_REGEN 0xFFFFFFFEu
#define O4_DRAW_PIDS 0x80000000u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_u53(uint32_t a, uint32_t b);

/* ------------------------------------------------------------------------ */
/* K0 from its integral representation K0(z) = int_0^inf exp(-z cosh t) dt  */
/* (z > 0).  The integrand is analytic and decays double-exponentially, so   */
/* the trapezoid rule with step 1/64 is exact to rounding; the sum stops     */
/* once z cosh t exceeds 750 (exp underflows).                               */
/* ------------------------------------------------------------------------ */
double orc4_k0(double z) {
  const double h = 1.0 / 64.0;
  double s = 0.5 * exp(-z);
  for (long i = 1;; ++i) {
    double t = h * (double)i;
    double e = z * cosh(t);
    if (e > 750.0) break;
    s += exp(-e);
  }
  return h * s;
}

typedef struct {
  double hbar, mass, dt;
  double Z, a, xc, lam;          /* charges, softening, nucleus position    */
  int nx, nk;                    /* cells per coordinate: nx^2 nk^2 in all   */
  double xmin, xmax, kmin, kmax; /* the same range for both electrons        */
  int ny, nkap;                  /* kernel table: y nodes x kappa cells      */
  long long n_alpha;
  unsigned long long seed;
} orc4_config;

typedef struct {
  double x1, x2, k1, k2, w;
  uint64_t pid;
} orc4_particle;

typedef struct {
  uint64_t pid, pid_plus, pid_minus;
  uint32_t step, j;
  double t, xe, kappa, factor;
  int32_t kill_plus, kill_minus;
  double xe2;
  int32_t comp, pad;
} orc4_event;

/* One kernel table (type 0: one-body, charge -Z; type 1: interaction, lam).
 * y_i = -Y + i dy (i < ny, dy = 2Y/(ny-1)); kappa_j = -K + (j + 1/2) dk
 * (j < nkap, dk = 2K/nkap).  v_ij = max(A_j sin(2 y_i kappa_j), 0),
 * S_ij = sum_{j' <= j} v_ij' (summed in order of j), xi_i = S_i,last dk. */
typedef struct {
  double Y, dy, inv_dy;
  double* A;  /* nkap */
  double* S;  /* ny x nkap */
  double* xi; /* ny */
  double gam; /* ceil(1024 max_i xi_i)/1024 */
} orc4_table;

/* O4_CAND: intervals in which a particle alive at their start has its first
 * event; O4_PAIRS0: those whose first event emits a pair. */
enum { O4_EVENTS = 0, O4_KILL_P, O4_KILL_M, O4_OUT_P, O4_OUT_M, O4_PSTEPS, O4_CAND, O4_PAIRS0,
       O4_LN = 8 };

typedef struct {
  orc4_config c;
  double hm, dtv, dx, dk, inv_dx, inv_dk, K, dkap, Gam;
  orc4_table tab[2];
  uint32_t key[2];
  orc4_particle *p, *q;
  long long n, cap, nq, capq;
  int* grid;
  long long step, epoch;
  int fresh;
  long long ledger[O4_LN];
  orc4_event* log;
  long long nlog, logcap;
  int log_on;
} orc4_state;

static void draw4(const orc4_state* s, uint64_t pid, uint32_t c2, uint32_t c3, uint32_t out[4]) {
  uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)(pid >> 32), c2, c3};
  orc_philox4x32_10(ctr, s->key, out);
}

static int push(orc4_particle** a, long long* n, long long* cap, orc4_particle v) {
  if (*n == *cap) {
    long long nc = *cap ? *cap * 2 : 1024;
    orc4_particle* b = (orc4_particle*)realloc(*a, (size_t)nc * sizeof(**a));
    if (!b) return -1;
    *a = b;
    *cap = nc;
  }
  (*a)[(*n)++] = v;
  return 0;
}

static int build_table(orc4_state* s, int type) {
  const orc4_config* c = &s->c;
  orc4_table* t = &s->tab[type];
  const int ny = c->ny, nk = c->nkap;
  /* y range: the histogram's x-width (one-body) or twice it (interaction) */
  t->Y = type == 0 ? (c->xmax - c->xmin) : 2.0 * (c->xmax - c->xmin);
  t->dy = 2.0 * t->Y / (double)(ny - 1);
  t->inv_dy = (double)(ny - 1) / (2.0 * t->Y);
  t->A = (double*)malloc((size_t)nk * sizeof(double));
  t->S = (double*)malloc((size_t)ny * (size_t)nk * sizeof(double));
  t->xi = (double*)malloc((size_t)ny * sizeof(double));
  if (!t->A || !t->S || !t->xi) return -1;
  const double q = type == 0 ? -c->Z : c->lam;
  const double pre = (4.0 * q) / (O4_PI * c->hbar); /* (2/(pi hbar)) q 2 */
  for (int j = 0; j < nk; ++j) {
    double kap = -s->K + ((double)j + 0.5) * s->dkap;
    t->A[j] = pre * orc4_k0(2.0 * c->a * fabs(kap));
  }
  double mx = 0.0;
  for (int i = 0; i < ny; ++i) {
    double y = -t->Y + (double)i * t->dy;
    double acc = 0.0;
    double* row = t->S + (size_t)i * nk;
    for (int j = 0; j < nk; ++j) {
      double kap = -s->K + ((double)j + 0.5) * s->dkap;
      double v = t->A[j] * sin(2.0 * y * kap);
      if (v > 0.0) acc += v;
      row[j] = acc;
    }
    t->xi[i] = acc * s->dkap;
    if (t->xi[i] > mx) mx = t->xi[i];
  }
  t->gam = ceil(1024.0 * mx) / 1024.0;
  return 0;
}

orc4_state* orc4_create(const orc4_config* c) {
  if (c->nx <= 0 || c->nk <= 0 || c->ny < 2 || c->nkap < 1 || !(c->xmax > c->xmin) ||
      !(c->kmax > c->kmin) || c->dt <= 0 || c->hbar <= 0 || c->mass <= 0 || !(c->a > 0) ||
      c->n_alpha <= 0)
    return NULL;
  orc4_state* s = (orc4_state*)calloc(1, sizeof(orc4_state));
  if (!s) return NULL;
  s->c = *c;
  s->hm = c->hbar / c->mass;
  s->dtv = c->dt * s->hm;
  s->dx = (c->xmax - c->xmin) / c->nx;
  s->dk = (c->kmax - c->kmin) / c->nk;
  s->inv_dx = c->nx / (c->xmax - c->xmin);
  s->inv_dk = c->nk / (c->kmax - c->kmin);
  s->K = c->kmax - c->kmin;
  s->dkap = 2.0 * s->K / (double)c->nkap;
  s->key[0] = (uint32_t)c->seed;
  s->key[1] = (uint32_t)(c->seed >> 32);
  long long nh = (long long)c->nx * c->nx * c->nk * c->nk;
  s->grid = (int*)calloc((size_t)nh, sizeof(int));
  if (!s->grid || build_table(s, 0) || build_table(s, 1)) {
    free(s->grid);
    for (int t = 0; t < 2; ++t) {
      free(s->tab[t].A);
      free(s->tab[t].S);
      free(s->tab[t].xi);
    }
    free(s);
    return NULL;
  }
  /* the rate of the clock: two one-body components and the interaction */
  s->Gam = 2.0 * s->tab[0].gam + s->tab[1].gam;
  if (!(s->Gam > 0)) s->Gam = 1.0; /* no potential: no pair is ever made */
  return s;
}

void orc4_destroy(orc4_state* s) {
  if (!s) return;
  free(s->p);
  free(s->q);
  free(s->grid);
  free(s->log);
  for (int t = 0; t < 2; ++t) {
    free(s->tab[t].A);
    free(s->tab[t].S);
    free(s->tab[t].xi);
  }
  free(s);
}

double orc4_gamma(const orc4_state* s, int type) { return s->tab[type].gam; }
double orc4_Gamma(const orc4_state* s) { return s->Gam; }
void orc4_enable_log(orc4_state* s, int on) { s->log_on = on; }

/* The table of one type: A (nkap), xi (ny) and the prefix sums S (ny*nkap). */
void orc4_get_table(const orc4_state* s, int type, double* A, double* xi, double* S) {
  const orc4_table* t = &s->tab[type];
  if (A) memcpy(A, t->A, (size_t)s->c.nkap * sizeof(double));
  if (xi) memcpy(xi, t->xi, (size_t)s->c.ny * sizeof(double));
  if (S) memcpy(S, t->S, (size_t)s->c.ny * (size_t)s->c.nkap * sizeof(double));
}

/* ------------------------------------------------------------------------ */
/* Initial data: the product of two Gaussian-wavepacket Wigner functions,    */
/* x_e ~ N(x0_e, sx^2), k_e ~ N(k0_e, 1/(4 sx^2)), sign +1; particle i has    */
/* pid = i; electron 1 from the draw (pid, INIT, 0), electron 2 from          */
/* (pid, INIT, 1), each by Box-Muller.                                       */
/* ------------------------------------------------------------------------ */
int orc4_init_gauss(orc4_state* s, long long n, double x01, double x02, double sx, double k01,
                    double k02) {
  double sk = 1.0 / (2.0 * sx);
  s->n = 0;
  for (long long i = 0; i < n; ++i) {
    orc4_particle p;
    double xs[2], ks[2];
    const double x0[2] = {x01, x02}, k0[2] = {k01, k02};
    for (int e = 0; e < 2; ++e) {
      uint32_t r[4];
      draw4(s, (uint64_t)i, O4_STEP_INIT, (uint32_t)e, r);
      double ua = orc_u53(r[0], r[1]);
      double ub = orc_u53(r[2], r[3]);
      double rad = sqrt(-2.0 * log1p(-ua));
      double th = O4_TWO_PI * ub;
      xs[e] = x0[e] + sx * (rad * cos(th));
      ks[e] = k0[e] + sk * (rad * sin(th));
    }
    p.x1 = xs[0];
    p.x2 = xs[1];
    p.k1 = ks[0];
    p.k2 = ks[1];
    p.w = 1.0;
    p.pid = (uint64_t)i;
    if (push(&s->p, &s->n, &s->cap, p)) return -1;
  }
  s->step = 0;
  s->epoch = 0;
  s->fresh = 0;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* One event j of a segment of pid in interval l at (x1e, x2e).  The draws   */
/* a = (pid, l, 1+2j) and b = (pid, l, 2+2j) give                            */
/*   ua = U53(a0,a1) acceptance and row, uk = U53(a2,a3) kick index,         */
/*   ug = U53(b0,b1) next gap, uc = b2 2^-32 component, uj = b3 2^-32        */
/*   position of the kick inside its kappa cell.                             */
/* Component m (0: y = x1-xc on k1; 1: y = x2-xc on k2; 2: y = x1-x2 on      */
/* (k1, -k2)) is the first with uc Gamma < gamma_0 + ... + gamma_m.  Its row */
/* position s = (y + Y)/dy (clamped to the mesh) splits into node i and      */
/* weight th; with g0 = (1-th) xi_i and g1 = th xi_{i+1} the pair is made     */
/* from row i if ua gamma_m < g0, from row i+1 if ua gamma_m < g0 + g1, and  */
/* not at all otherwise (probability xi_h(y)/gamma_m, xi_h the linear        */
/* interpolant; the row choice makes the kick law the interpolant of the     */
/* rows' laws).  The kick is kappa_j + (uj - 1/2) dkappa for the first j      */
/* with S_rj > uk S_r,last.  Returns 1 if a pair is made.                    */
/* ------------------------------------------------------------------------ */
static int event4(const orc4_state* s, uint64_t pid, uint32_t l, uint32_t j, double x1e,
                  double x2e, int* comp, double* kap, double* prob, double* gap) {
  uint32_t a[4], b[4];
  draw4(s, pid, l, 1u + 2u * j, a);
  draw4(s, pid, l, 2u + 2u * j, b);
  double ua = orc_u53(a[0], a[1]);
  double uk = orc_u53(a[2], a[3]);
  double ug = orc_u53(b[0], b[1]);
  double uc = (double)b[2] * (1.0 / 4294967296.0);
  double uj = (double)b[3] * (1.0 / 4294967296.0);
  *gap = -log1p(-ug) / s->Gam;
  double g_ne = s->tab[0].gam, g_ee = s->tab[1].gam;
  double v = uc * s->Gam;
  int m = v < g_ne ? 0 : (v < 2.0 * g_ne ? 1 : 2);
  *comp = m;
  const orc4_table* t = &s->tab[m == 2 ? 1 : 0];
  double y = m == 0 ? x1e - s->c.xc : (m == 1 ? x2e - s->c.xc : x1e - x2e);
  double g = m == 2 ? g_ee : g_ne;
  double sp = (y + t->Y) * t->inv_dy;
  long i;
  double th;
  if (!(sp > 0.0)) {
    i = 0;
    th = 0.0;
  } else if (sp >= (double)(s->c.ny - 1)) {
    i = s->c.ny - 2;
    th = 1.0;
  } else {
    i = (long)floor(sp);
    th = sp - (double)i;
  }
  double g0 = (1.0 - th) * t->xi[i];
  double g1 = th * t->xi[i + 1];
  *prob = g > 0.0 ? (g0 + g1) / g : 0.0;
  double va = ua * g;
  long r;
  if (va < g0) r = i;
  else if (va < g0 + g1) r = i + 1;
  else return 0;
  const double* row = t->S + (size_t)r * s->c.nkap;
  double target = uk * row[s->c.nkap - 1];
  long lo = 0, hi = s->c.nkap - 1; /* first j with row[j] > target */
  while (lo < hi) {
    long mid = (lo + hi) / 2;
    if (row[mid] > target) hi = mid; else lo = mid + 1;
  }
  double kj = -s->K + ((double)lo + 0.5) * s->dkap;
  *kap = kj + (uj - 0.5) * s->dkap;
  return 1;
}

int orc4_event_outcome(const orc4_state* s, uint64_t pid, uint32_t l, uint32_t j, double x1e,
                       double x2e, int* comp, double* kappa, double* prob, double* gap) {
  *kappa = 0.0;
  return event4(s, pid, l, j, x1e, x2e, comp, kappa, prob, gap);
}

static int kin(const orc4_state* s, double k) { return k >= s->c.kmin && k < s->c.kmax; }

/* The part of interval l of a particle from time `to` (Alg. 1 with the     */
/* draws above; offspring recurse from their birth time).                   */
static int segment4(orc4_state* s, double x1o, double x2o, double to, double k1, double k2,
                    double w, uint64_t pid, uint32_t l, int is_root) {
  const orc4_config* c = &s->c;
  uint32_t r[4];
  draw4(s, pid, l, 0u, r);
  double u0 = orc_u53(r[0], r[1]);
  double t = to + (-log1p(-u0) / s->Gam);
  uint32_t j = 0;
  if (is_root && t < c->dt) s->ledger[O4_CAND] += 1;
  while (t < c->dt) {
    double x1e = x1o + k1 * ((t - to) * s->hm);
    double x2e = x2o + k2 * ((t - to) * s->hm);
    int m;
    double kap, prob, gap;
    if (event4(s, pid, l, j, x1e, x2e, &m, &kap, &prob, &gap)) {
      uint32_t h[4];
      draw4(s, pid, l, O4_DRAW_PIDS | j, h);
      uint64_t pid_p = (1ull << 63) | ((((uint64_t)h[1] << 32) | (uint64_t)h[0]) >> 1);
      uint64_t pid_m = (1ull << 63) | ((((uint64_t)h[3] << 32) | (uint64_t)h[2]) >> 1);
      /* + child at k + kappa e_m, - child at k - kappa e_m, with
       * e_0 = (1, 0), e_1 = (0, 1), e_2 = (1, -1) */
      double kp1 = k1, kp2 = k2, km1 = k1, km2 = k2;
      if (m == 0) {
        kp1 = k1 + kap;
        km1 = k1 - kap;
      } else if (m == 1) {
        kp2 = k2 + kap;
        km2 = k2 - kap;
      } else {
        kp1 = k1 + kap;
        kp2 = k2 - kap;
        km1 = k1 - kap;
        km2 = k2 + kap;
      }
      int kill_p = !(kin(s, kp1) && kin(s, kp2));
      int kill_m = !(kin(s, km1) && kin(s, km2));
      s->ledger[O4_EVENTS] += 1;
      if (is_root && j == 0) s->ledger[O4_PAIRS0] += 1;
      double wp = w, wm = -w;
      if (kill_p) { if (wp > 0) s->ledger[O4_KILL_P] += 1; else s->ledger[O4_KILL_M] += 1; }
      if (kill_m) { if (wm > 0) s->ledger[O4_KILL_P] += 1; else s->ledger[O4_KILL_M] += 1; }
      if (s->log_on) {
        if (s->nlog == s->logcap) {
          long long nc = s->logcap ? s->logcap * 2 : 1024;
          orc4_event* b2 = (orc4_event*)realloc(s->log, (size_t)nc * sizeof(orc4_event));
          if (!b2) return -1;
          s->log = b2;
          s->logcap = nc;
        }
        orc4_event e;
        memset(&e, 0, sizeof(e));
        e.pid = pid;
        e.pid_plus = pid_p;
        e.pid_minus = pid_m;
        e.step = l;
        e.j = j;
        e.t = t;
        e.xe = x1e;
        e.xe2 = x2e;
        e.kappa = kap;
        e.factor = prob;
        e.kill_plus = kill_p;
        e.kill_minus = kill_m;
        e.comp = m;
        s->log[s->nlog++] = e;
      }
      if (!kill_p && segment4(s, x1e, x2e, t, kp1, kp2, wp, pid_p, l, 0)) return -1;
      if (!kill_m && segment4(s, x1e, x2e, t, km1, km2, wm, pid_m, l, 0)) return -1;
    }
    t += gap;
    ++j;
  }
  orc4_particle out;
  if (is_root) {
    out.x1 = x1o + k1 * s->dtv;
    out.x2 = x2o + k2 * s->dtv;
  } else {
    out.x1 = x1o + k1 * ((c->dt - to) * s->hm);
    out.x2 = x2o + k2 * ((c->dt - to) * s->hm);
  }
  out.k1 = k1;
  out.k2 = k2;
  out.w = w;
  out.pid = pid;
  return push(&s->q, &s->nq, &s->capq, out);
}

int orc4_step(orc4_state* s, int nsteps) {
  for (int it = 0; it < nsteps; ++it) {
    uint32_t l = (uint32_t)s->step;
    s->nq = 0;
    s->ledger[O4_PSTEPS] += s->n;
    for (long long i = 0; i < s->n; ++i) {
      orc4_particle p = s->p[i];
      if (segment4(s, p.x1, p.x2, 0.0, p.k1, p.k2, p.w, p.pid, l, 1)) return -1;
    }
    orc4_particle* t = s->p;
    s->p = s->q;
    s->q = t;
    long long tc = s->cap;
    s->cap = s->capq;
    s->capq = tc;
    s->n = s->nq;
    s->step += 1;
    s->fresh = 0;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Histogram on the 4D mesh: cell nu = ((ix1 nx + ix2) nk + ik1) nk + ik2.   */
/* ------------------------------------------------------------------------ */
static double binx(const orc4_state* s, double x) { return floor((x - s->c.xmin) * s->inv_dx); }
static double bink(const orc4_state* s, double k) { return floor((k - s->c.kmin) * s->inv_dk); }

static int cell4(const orc4_state* s, const orc4_particle* p, long long* nu) {
  double f[4] = {binx(s, p->x1), binx(s, p->x2), bink(s, p->k1), bink(s, p->k2)};
  double lim[4] = {(double)s->c.nx, (double)s->c.nx, (double)s->c.nk, (double)s->c.nk};
  for (int d = 0; d < 4; ++d)
    if (!(f[d] >= 0.0 && f[d] < lim[d])) return 0;
  *nu = (((long long)f[0] * s->c.nx + (long long)f[1]) * s->c.nk + (long long)f[2]) * s->c.nk +
        (long long)f[3];
  return 1;
}

static void bin4(orc4_state* s) {
  long long nh = (long long)s->c.nx * s->c.nx * s->c.nk * s->c.nk;
  memset(s->grid, 0, (size_t)nh * sizeof(int));
  for (long long i = 0; i < s->n; ++i) {
    long long nu;
    if (cell4(s, &s->p[i], &nu)) {
      s->grid[nu] += s->p[i].w > 0 ? 1 : -1;
    } else {
      if (s->p[i].w > 0) s->ledger[O4_OUT_P] += 1; else s->ledger[O4_OUT_M] += 1;
    }
  }
}

static double fix_into(double x, double lo, double inv, double idx) {
  while (floor((x - lo) * inv) > idx) x = nextafter(x, -INFINITY);
  while (floor((x - lo) * inv) < idx) x = nextafter(x, INFINITY);
  return x;
}

/* Alg. 3 without rounding on the 4D mesh: particle j (cells in order) has
 * pid = (epoch << 40) | j, x offsets U53 pairs of (pid, REGEN, 0) and k
 * offsets of (pid, REGEN, 1). */
static int regenerate4(orc4_state* s) {
  const orc4_config* c = &s->c;
  long long nh = (long long)c->nx * c->nx * c->nk * c->nk;
  s->n = 0;
  uint64_t j = 0;
  for (long long nu = 0; nu < nh; ++nu) {
    int cnt = s->grid[nu];
    if (cnt == 0) continue;
    long long ik2 = nu % c->nk, r1 = nu / c->nk;
    long long ik1 = r1 % c->nk, r2 = r1 / c->nk;
    long long ix2 = r2 % c->nx, ix1 = r2 / c->nx;
    long long m = cnt > 0 ? cnt : -(long long)cnt;
    double sign = cnt > 0 ? 1.0 : -1.0;
    for (long long r = 0; r < m; ++r, ++j) {
      uint64_t pid = ((uint64_t)s->epoch << 40) | j;
      uint32_t h[4], g[4];
      draw4(s, pid, O4_STEP_REGEN, 0u, h);
      draw4(s, pid, O4_STEP_REGEN, 1u, g);
      orc4_particle p;
      p.x1 = fix_into(c->xmin + ((double)ix1 + orc_u53(h[0], h[1])) * s->dx, c->xmin, s->inv_dx,
                      (double)ix1);
      p.x2 = fix_into(c->xmin + ((double)ix2 + orc_u53(h[2], h[3])) * s->dx, c->xmin, s->inv_dx,
                      (double)ix2);
      p.k1 = fix_into(c->kmin + ((double)ik1 + orc_u53(g[0], g[1])) * s->dk, c->kmin, s->inv_dk,
                      (double)ik1);
      p.k2 = fix_into(c->kmin + ((double)ik2 + orc_u53(g[2], g[3])) * s->dk, c->kmin, s->inv_dk,
                      (double)ik2);
      p.w = sign;
      p.pid = pid;
      if (push(&s->p, &s->n, &s->cap, p)) return -1;
    }
  }
  return 0;
}

int orc4_annihilate(orc4_state* s) {
  if (s->fresh) return 0;
  s->epoch += 1;
  bin4(s);
  if (regenerate4(s)) return -1;
  s->fresh = 1;
  return 0;
}

long long orc4_count(const orc4_state* s) { return s->n; }
long long orc4_epoch(const orc4_state* s) { return s->epoch; }

void orc4_get_particles(const orc4_state* s, double* x1, double* x2, double* k1, double* k2,
                        double* w, uint64_t* pid) {
  for (long long i = 0; i < s->n; ++i) {
    x1[i] = s->p[i].x1;
    x2[i] = s->p[i].x2;
    k1[i] = s->p[i].k1;
    k2[i] = s->p[i].k2;
    w[i] = s->p[i].w;
    pid[i] = s->p[i].pid;
  }
}

void orc4_get_grid(const orc4_state* s, int* grid) {
  long long nh = (long long)s->c.nx * s->c.nx * s->c.nk * s->c.nk;
  memcpy(grid, s->grid, (size_t)nh * sizeof(int));
}

void orc4_get_ledger(const orc4_state* s, long long* out) {
  memcpy(out, s->ledger, sizeof(s->ledger));
}

long long orc4_log_count(const orc4_state* s) { return s->nlog; }
void orc4_get_log(const orc4_state* s, orc4_event* out) {
  memcpy(out, s->log, (size_t)s->nlog * sizeof(orc4_event));
}
long long orc4_event_size(void) { return (long long)sizeof(orc4_event); }

/* Observables of electron 1 (Eq. estimator): the reduced Wigner function
 * f1(x1, k1) = sum_{x2, k2 cells} c / (N_alpha dx dk) (nx*nk), its spatial
 * marginal sum_{k1} / (N_alpha dx) (nx) and sum over cells with x1-centre
 * > 0 of c / N_alpha. */
void orc4_observables(const orc4_state* s, const int* counts, double* f1, double* marg,
                      double* right) {
  const orc4_config* c = &s->c;
  const long long nx = c->nx, nk = c->nk;
  double na = (double)c->n_alpha;
  long long* red = (long long*)calloc((size_t)(nx * nk), sizeof(long long));
  if (!red) return;
  for (long long ix1 = 0; ix1 < nx; ++ix1)
    for (long long ix2 = 0; ix2 < nx; ++ix2)
      for (long long ik1 = 0; ik1 < nk; ++ik1)
        for (long long ik2 = 0; ik2 < nk; ++ik2)
          red[ix1 * nk + ik1] += counts[((ix1 * nx + ix2) * nk + ik1) * nk + ik2];
  long long tot = 0;
  for (long long ix = 0; ix < nx; ++ix) {
    long long col = 0;
    for (long long ik = 0; ik < nk; ++ik) {
      long long v = red[ix * nk + ik];
      col += v;
      if (f1) f1[ix * nk + ik] = (double)v / (na * s->dx * s->dk);
    }
    if (marg) marg[ix] = (double)col / (na * s->dx);
    double centre = c->xmin + ((double)ix + 0.5) * s->dx;
    if (centre > 0.0) tot += col;
  }
  if (right) *right = (double)tot / na;
  free(red);
}
