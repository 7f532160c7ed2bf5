/*
 * dies_oracle.c -- serial FP64 oracle of the immediate re-emission (IRE)
 * Monte Carlo method for spherically symmetric dust clouds (Juvela 2024,
 * "DIES", Sect. 2 and Sect. 2.2).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference against
 * which the CUDA library is checked.  Only the test suite, the package smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, constant table or helper with the CUDA library; the two only
 * consume the same seeded input arrays.
 *
 * What it computes (one package at a time, everything in double precision,
 * 3-D position and direction vectors as in Sect. 2.1):
 *   - sources (Sect. 2.1): isotropic external field entering at (0,0,-R) with
 *     mu = sqrt(u) (Eqs. 2-3) and a central point source with mu uniform in
 *     [-1,1]; the luminosity of each source is split over N equal packages;
 *   - free paths tau_S = -ln u1, tau_A = -ln u2 drawn independently (Eq. 1)
 *     and consumed cell by cell (Eq. 4);
 *   - scattering by the Henyey-Greenstein phase function (the HG form quoted
 *     in Sect. 2.2.1, Eq. 6) when tau_S runs out first;
 *   - absorption when tau_A runs out first: the package energy is added to
 *     the cell, the cell temperature is updated immediately, and the same
 *     energy is re-emitted isotropically at a frequency drawn from the
 *     difference between the cell emission spectra at the new and old
 *     temperatures (Sect. 2.1);
 *   - direction weighting of background packages, mu = u^k_bg with weight
 *     2 k_bg mu^(2-1/k_bg) (Sect. 2.2.1, Eq. 5);
 *   - forced first interaction (Sect. 2.2.2, Eqs. 9-12), with the extinction
 *     optical depth (absorption + scattering) as the forced variable, or
 *     (the stronger variant named at the end of Sect. 2.2.2) the optical
 *     depth of absorption only;
 *   - direction weighting of re-emission (Sect. 2.2.1, Eq. 6): the new
 *     direction from a Henyey-Greenstein function of parameter g_E about the
 *     reference direction (towards the centre for packages of the external
 *     field, away from it for the point source), weight = isotropic pdf /
 *     HG pdf;
 *   - direction weighting of scattering (Sect. 2.2.1, Eq. 7): the new
 *     direction from an HG function of parameter g_S about the reference
 *     direction, weight = dust HG pdf of the scattering angle / HG(g_S) pdf
 *     of the angle to the reference direction;
 *   - optionally, re-emission from a point drawn uniformly over the volume of
 *     the absorbing cell instead of the absorption point (the test variant
 *     of Sect. 4): r^3 uniform between the cell's inner and outer r^3, the
 *     angular position kept (irrelevant by symmetry);
 *   - free-path weighting (Sect. 2.2.2, Eq. 8): tau = -ln(u) / k with weight
 *     e^(tau (k - 1)) / k, separately for absorption (k_A) and scattering
 *     (k_S); optionally k_A per cell, linear in log density from k_A_lo at the
 *     lowest cell density to k_A_hi at the highest;
 *   - the weight floor: a package whose weight has fallen ten orders of
 *     magnitude is terminated (Sect. 2.2.1).
 *
 * Readings where the paper is silent (each listed with its reason in the
 * design notes): packages carry one of F discrete frequency bins and every
 * spectral integral is sum_k f(nu_k) dnu_k with log-midpoint weights; the
 * temperature is the exact FP64 root of 4 pi V rho L_u^2 sum_k kabs_k
 * B_k(T) dnu_k = E (no lookup table); the difference spectrum is the exact
 * kabs_k [B_k(T_new) - B_k(T_old)] dnu_k; the direct-escape fraction
 * e^-tau0 of a forced package is tallied in the escaping SED so that energy
 * is conserved exactly.  Forcing on the absorption depth alone: the
 * scattering clock keeps its plain draw; only when it outlasts the whole
 * first ray is the absorption forced inside the ray (weight 1 - e^-tau_A0,
 * e^-tau_A0 tallied as a direct escape), otherwise the first flight is
 * unforced -- this keeps the estimator unbiased with scattering.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw 2011) keyed by
 * the 64-bit seed, counter (package lo, package hi, block index,
 * model id ^ source id << 24).  Each block of four 32-bit words gives two
 * doubles u = (m + 1/2) 2^-52 with m the top 52 bits of a word pair, so
 * 0 < u < 1 exactly.  Blocks per event: injection {u_freq, u_mu},
 * {u_tauS, u_tauA}; forced first interaction {u_int, u_type}; scattering
 * {u_mu_s, u_phi}, {u_tauS, u_tauA}; absorption {u_e, u_nu}, {u_mu, u_phi},
 * {u_tauS, u_tauA}.  u_e is reserved for table-based temperature updates and
 * is drawn but unused here.  With the re-emission point randomised, one more
 * block {u_r, unused} follows {u_e, u_nu}.  The weighted directions use the same blocks:
 * {u_mu, u_phi} give the cosine to the reference direction and the azimuth
 * about it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
/* CGS constants (exact values of the 2019 SI definitions). */
#define ORC_H  6.62607015e-27  /* erg s */
#define ORC_KB 1.380649e-16    /* erg / K */
#define ORC_C  2.99792458e10   /* cm / s */

#define ORC_MAX_FREQ 4096

enum { ORC_MODE_IRE = 0, ORC_MODE_FROZEN = 1, ORC_MODE_FROZEN_TERMINAL = 2 };
enum { ORC_EV_INJECT = 0, ORC_EV_CROSS = 1, ORC_EV_SCATTER = 2, ORC_EV_ABSORB = 3 };

/* indices of the statistics vector */
enum {
  ST_INJECTED = 0, ST_ESCAPED, ST_ABSORB, ST_SCATTER, ST_CROSS, ST_KILL_WEIGHT, ST_KILL_CAP,
  ST_CLAMP_HI, ST_E_INJECTED, ST_E_ESCAPED, ST_E_LOST, ST_E_DIRECT, ST_FORCED, ST_COUNT
};

typedef struct {
  int32_t n_cells;
  int32_t n_freq;
  const double *radii;      /* n_cells + 1, strictly increasing, radii[0] >= 0 */
  const double *rho;        /* n_cells, >= 0 */
  double length_unit_cm;    /* cm per length unit of radii; kappa*rho is per length unit */
  const double *freq;       /* n_freq, Hz, strictly increasing */
  const double *kabs;       /* n_freq */
  const double *ksca;       /* n_freq */
  const double *g;          /* n_freq, HG asymmetry */
  const double *J_ext;      /* n_freq isotropic intensity, or NULL */
  double L_point;           /* erg/s, 0 = no point source */
  const double *point_spec; /* n_freq L_nu shape, or NULL */
  double k_bg;              /* 0.5 = unweighted */
  int32_t ffi;              /* forced first interaction: 0 off, 1 on tau_ext, 2 on tau_A */
  double g_E;               /* re-emission direction weighting (Eq. 6); 0 = off */
  int32_t scat_w;           /* scattering direction weighting (Eq. 7) on */
  double g_S;               /* its HG parameter */
  double k_A, k_S;          /* free-path weighting (Eq. 8); 1 = off */
  int32_t kA_rho;           /* density-dependent k_A */
  double kA_lo, kA_hi;      /* k_A at the lowest and at the highest cell density */
  int32_t remit_random;     /* re-emit from a point uniform over the cell volume */
  double T_min, T_max;      /* reporting range of the temperatures */
  uint32_t model_id;
  uint64_t max_events;      /* per package; 0 = 1e8 */
} orc_model;

/* ------------------------------------------------------------------ RNG */

/* Philox4x32 with 10 rounds: each round multiplies words 0 and 2 by the two
 * Philox constants, swaps in the xor of the high halves with the other words
 * and the round key, and the key is bumped by the two Weyl increments between
 * rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform double in (0,1) from two 32-bit words: m = top 52 bits, u = (m+1/2) 2^-52. */
double orc_u01(uint32_t a, uint32_t b)
{
  uint64_t m = ((uint64_t)a << 20) | (uint64_t)(b >> 12);
  return ((double)m + 0.5) * 0x1p-52;
}

typedef struct {
  uint32_t key[2];
  uint32_t ctr[4];
} orc_stream;

static void stream_init(orc_stream *s, uint64_t seed, uint64_t pkg, uint32_t model_id, uint32_t source)
{
  s->key[0] = (uint32_t)seed;
  s->key[1] = (uint32_t)(seed >> 32);
  s->ctr[0] = (uint32_t)pkg;
  s->ctr[1] = (uint32_t)(pkg >> 32);
  s->ctr[2] = 0;
  s->ctr[3] = model_id ^ (source << 24);
}

static void draw2(orc_stream *s, double *ua, double *ub)
{
  uint32_t o[4];
  orc_philox4x32_10(s->ctr, s->key, o);
  s->ctr[2] += 1;
  *ua = orc_u01(o[0], o[1]);
  *ub = orc_u01(o[2], o[3]);
}

/* ------------------------------------------------------- spectra, tables */

/* Planck intensity B_nu(T), erg/s/cm^2/Hz/sr. */
double orc_planck(double nu, double T)
{
  if (!(T > 0.0)) return 0.0;
  double x = ORC_H * nu / (ORC_KB * T);
  if (x > 700.0) return 0.0;
  return 2.0 * ORC_H * nu * nu * nu / (ORC_C * ORC_C) / expm1(x);
}

/* dB_nu/dT */
double orc_dplanck_dT(double nu, double T)
{
  if (!(T > 0.0)) return 0.0;
  double x = ORC_H * nu / (ORC_KB * T);
  if (x > 700.0) return 0.0;
  double em1 = expm1(x);
  double B = 2.0 * ORC_H * nu * nu * nu / (ORC_C * ORC_C) / em1;
  return B * x * (em1 + 1.0) / (em1 * T);
}

/* Quadrature weights dnu_k = nu_k * (width of bin k in ln nu): half the
 * distance to the neighbours in ln nu inside the grid, the full distance to
 * the single neighbour at the two ends.  On a log-uniform grid every weight
 * is nu_k * dln(nu). */
int orc_freq_weights(int F, const double *nu, double *dnu)
{
  if (F < 2) return -1;
  for (int k = 0; k < F; ++k) {
    double w;
    if (k == 0) w = log(nu[1]) - log(nu[0]);
    else if (k == F - 1) w = log(nu[F - 1]) - log(nu[F - 2]);
    else w = 0.5 * (log(nu[k + 1]) - log(nu[k - 1]));
    dnu[k] = nu[k] * w;
  }
  return 0;
}

/* Emission per unit (4 pi rho V L_u^2): Lambda(T) = sum_k kabs_k B_k(T) dnu_k. */
double orc_emission(int F, const double *nu, const double *dnu, const double *kabs, double T)
{
  double s = 0.0;
  for (int k = 0; k < F; ++k) s += kabs[k] * orc_planck(nu[k], T) * dnu[k];
  return s;
}

static double emission_and_derivative(int F, const double *nu, const double *dnu, const double *kabs,
                                      double T, double *dLdT)
{
  double s = 0.0, d = 0.0;
  for (int k = 0; k < F; ++k) {
    double x = ORC_H * nu[k] / (ORC_KB * T);
    if (x > 700.0) continue;
    double em1 = expm1(x);
    double B = 2.0 * ORC_H * nu[k] * nu[k] * nu[k] / (ORC_C * ORC_C) / em1;
    s += kabs[k] * B * dnu[k];
    d += kabs[k] * B * x * (em1 + 1.0) / (em1 * T) * dnu[k];
  }
  *dLdT = d;
  return s;
}

#define ORC_T_LO 1e-2
#define ORC_T_HI 1e6

/* Temperature T with Lambda(T) = e, given Lambda at the bracket ends
 * [1e-2 K, 1e6 K]: safeguarded Newton iteration on ln Lambda(T) = ln e in the
 * variable ln T, started from T_guess, falling back to bisection whenever a
 * Newton step leaves the current bracket.  e <= 0 gives 0; e beyond the
 * bracket values gives the bracket end. */
static double solve_temperature(int F, const double *nu, const double *dnu, const double *kabs, double e,
                                double T_guess, double L_lo, double L_hi)
{
  if (!(e > 0.0)) return 0.0;
  if (e <= L_lo) return ORC_T_LO;
  if (e >= L_hi) return ORC_T_HI;
  double d;
  double lo = log(ORC_T_LO), hi = log(ORC_T_HI);
  double le = log(e);
  double x = (T_guess > ORC_T_LO && T_guess < ORC_T_HI) ? log(T_guess) : 0.5 * (lo + hi);
  for (int it = 0; it < 300; ++it) {
    double T = exp(x);
    double L = emission_and_derivative(F, nu, dnu, kabs, T, &d);
    double f = (L > 0.0) ? log(L) - le : -1e300;
    if (f > 0.0) hi = x; else lo = x;
    double xn;
    if (L > 0.0 && d > 0.0) {
      xn = x - f / (T * d / L);   /* d lnL / d lnT = T L' / L */
      if (fabs(xn - x) < 1e-13) { x = xn; break; }
    } else {
      xn = 0.5 * (lo + hi);
    }
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    if (hi - lo < 1e-15) { x = xn; break; }
    x = xn;
  }
  return exp(x);
}

double orc_temperature(int F, const double *nu, const double *dnu, const double *kabs, double e,
                       double T_guess)
{
  double L_lo = orc_emission(F, nu, dnu, kabs, ORC_T_LO);
  double L_hi = orc_emission(F, nu, dnu, kabs, ORC_T_HI);
  return solve_temperature(F, nu, dnu, kabs, e, T_guess, L_lo, L_hi);
}

/* Henyey-Greenstein scattering cosine by inversion of the HG cumulative
 * distribution (the HG form of Sect. 2.2.1, Eq. 6); |g| < 1e-6 is isotropic. */
double orc_hg_mu(double g, double u)
{
  if (fabs(g) < 1e-6) return 2.0 * u - 1.0;
  double t = (1.0 - g * g) / (1.0 - g + 2.0 * g * u);
  double mu = (1.0 + g * g - t * t) / (2.0 * g);
  if (mu > 1.0) mu = 1.0;
  if (mu < -1.0) mu = -1.0;
  return mu;
}

/* Henyey-Greenstein density of the cosine mu without the common factor
 * 1/2: (1 - g^2) / (1 + g^2 - 2 g mu)^(3/2) (Eq. 6); 1 for g = 0. */
double orc_hg_pdf2(double g, double mu)
{
  double q = 1.0 + g * g - 2.0 * g * mu;
  return (1.0 - g * g) / (q * sqrt(q));
}

/* Radius of a point uniform over the volume of the shell [ri, ro]. */
double orc_shell_radius(double ri, double ro, double u)
{
  double a = ri * ri * ri, b = ro * ro * ro;
  return cbrt(a + u * (b - a));
}

/* Free-path weight of Eq. 8 for a path tau drawn from k e^(-k tau). */
double orc_path_weight(double k, double tau)
{
  return exp(tau * (k - 1.0)) / k;
}

/* smallest k with cdf[k] >= u (cdf[F-1] == 1) */
static int sample_cdf(int F, const double *cdf, double u)
{
  for (int k = 0; k < F; ++k)
    if (cdf[k] >= u) return k;
  return F - 1;
}

static void make_cdf(int F, const double *p, double *cdf)
{
  double s = 0.0;
  for (int k = 0; k < F; ++k) { s += p[k]; cdf[k] = s; }
  for (int k = 0; k < F; ++k) cdf[k] = (s > 0.0) ? cdf[k] / s : (double)(k + 1) / F;
  cdf[F - 1] = 1.0;
}

/* ---------------------------------------------------------- 3-D vectors */

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void normalise3(double *a)
{
  double n = sqrt(dot3(a, a));
  a[0] /= n; a[1] /= n; a[2] /= n;
}

/* Two unit vectors e1, e2 completing the unit vector a to a right-handed
 * orthonormal frame; e1 lies in the plane of a and ref when they are not
 * parallel (ref need not be normalised; NULL or parallel -> any). */
static void frame(const double *a, const double *ref, double *e1, double *e2)
{
  double t[3] = {0.0, 0.0, 0.0};
  double n = 0.0;
  if (ref) {
    double ra = dot3(ref, a);
    for (int i = 0; i < 3; ++i) t[i] = ref[i] - ra * a[i];
    n = sqrt(dot3(t, t));
    double rn = sqrt(dot3(ref, ref));
    if (!(n > 1e-300) || n < 1e-14 * rn) n = 0.0;
  }
  if (n == 0.0) {
    /* any perpendicular: cross with the axis least aligned with a */
    double ax[3] = {0.0, 0.0, 0.0};
    int m = 0;
    if (fabs(a[1]) < fabs(a[m])) m = 1;
    if (fabs(a[2]) < fabs(a[m])) m = 2;
    ax[m] = 1.0;
    double ra = dot3(ax, a);
    for (int i = 0; i < 3; ++i) t[i] = ax[i] - ra * a[i];
    n = sqrt(dot3(t, t));
  }
  for (int i = 0; i < 3; ++i) e1[i] = t[i] / n;
  e2[0] = a[1] * e1[2] - a[2] * e1[1];
  e2[1] = a[2] * e1[0] - a[0] * e1[2];
  e2[2] = a[0] * e1[1] - a[1] * e1[0];
}

/* ------------------------------------------------------------ the model */

typedef struct {
  const orc_model *M;
  int n, F;
  double R;
  double dnu[ORC_MAX_FREQ];
  double cdf_src[2][ORC_MAX_FREQ];
  double eps[2];           /* package energy per source, erg/s */
  int active[2];
  double *mass;            /* n: 4 pi rho V L_u^2, so that E = mass * Lambda(T) */
  double *kA;              /* n: absorption free-path weighting factor per cell */
  double kA_void;          /* ... in the central void (and empty cells) */
  double *E;               /* n: absorbed energy */
  double *T;               /* n: current temperature */
  double *Bcur;            /* n*F: kabs_k B_k(T_cur) dnu_k for the cell */
  double *cdf_frozen;      /* n*F */
  double Lmax;             /* Lambda(T_max): clamp counter threshold */
  double L_lo, L_hi;       /* Lambda at the ends of the root bracket */
  int mode;
  double *sed;
  double *st;
  uint64_t max_events;
} orc_ctx;

typedef struct {
  double x[3], d[3];
  int cell;                /* -1 = central void, n = outside */
  int f;
  double w;                /* weight relative to an unweighted package */
  double tauA, tauS;
  uint32_t nev[3];         /* scatter, absorb, cross */
  uint64_t hash;
  uint64_t events;
} orc_pkg;

#define FNV_OFFSET 0xcbf29ce484222325ULL
#define FNV_PRIME 0x100000001b3ULL

/* Path record of one event: 32-bit word event | (cell+1) << 3 | freq << 24,
 * folded into a 64-bit FNV-1a hash byte by byte (little endian). */
static void record(orc_pkg *p, int ev, int cell, int f)
{
  uint32_t w = (uint32_t)ev | ((uint32_t)(cell + 1) << 3) | ((uint32_t)f << 24);
  for (int b = 0; b < 4; ++b) {
    p->hash ^= (uint64_t)((w >> (8 * b)) & 0xffu);
    p->hash *= FNV_PRIME;
  }
}

/* Distance along the ray to the boundary through which the package leaves
 * its current cell; *next = the cell entered there (n = outside, -1 = the
 * central void).  Inside the void only the sphere radii[0] is a boundary. */
static double boundary_distance(const orc_ctx *C, const double *x, const double *d, int cell, int *next)
{
  const double *r = C->M->radii;
  double rr = dot3(x, x), b = dot3(x, d);
  if (cell >= 0 && r[cell] > 0.0 && b < 0.0) {
    double ri2 = r[cell] * r[cell];
    double disc = b * b - (rr - ri2);
    if (disc > 0.0) {
      double l = (rr - ri2) / (-b + sqrt(disc));  /* = -b - sqrt(disc), cancellation-free */
      *next = cell - 1;
      return l > 0.0 ? l : 0.0;
    }
  }
  double ro = (cell >= 0) ? r[cell + 1] : r[0];
  double c = rr - ro * ro;
  double disc = b * b - c;
  if (disc < 0.0) disc = 0.0;
  double l = (b <= 0.0) ? (-b + sqrt(disc)) : (-c / (b + sqrt(disc)));
  *next = (cell >= 0) ? cell + 1 : 0;
  return l > 0.0 ? l : 0.0;
}

static double kabs_cell(const orc_ctx *C, int cell, int f)
{
  return (cell >= 0) ? C->M->kabs[f] * C->M->rho[cell] : 0.0;
}

static double ksca_cell(const orc_ctx *C, int cell, int f)
{
  return (cell >= 0) ? C->M->ksca[f] * C->M->rho[cell] : 0.0;
}

static void move(orc_pkg *p, double l)
{
  for (int i = 0; i < 3; ++i) p->x[i] += l * p->d[i];
}

static void escape(orc_ctx *C, orc_pkg *p, int s)
{
  double e = p->w * C->eps[s];
  C->sed[p->f] += e;
  C->st[ST_ESCAPED] += 1.0;
  C->st[ST_E_ESCAPED] += e;
}

static void lose(orc_ctx *C, orc_pkg *p, int s, int why)
{
  C->st[why] += 1.0;
  C->st[ST_E_LOST] += p->w * C->eps[s];
}

/* Reference direction of the weighted direction distributions (Sect.
 * 2.2.1): towards the centre for packages of the external field (s = 0),
 * away from it for the point source (s = 1). */
static void reference_direction(const orc_pkg *p, int s, double *ref)
{
  double xr = sqrt(dot3(p->x, p->x));
  double rhat[3] = {0.0, 0.0, 1.0};
  if (xr > 0.0)
    for (int i = 0; i < 3; ++i) rhat[i] = p->x[i] / xr;
  for (int i = 0; i < 3; ++i) ref[i] = (s == 0) ? -rhat[i] : rhat[i];
}

/* Both free paths (Eq. 1) from one block, each weighted by Eq. 8 when its k
 * differs from 1; k_A is that of the package's current cell. */
static void draw_paths(orc_ctx *C, orc_pkg *p, orc_stream *rs)
{
  double u1, u2;
  draw2(rs, &u1, &u2);
  double kS = C->M->k_S;
  double kA = (p->cell >= 0 && p->cell < C->n) ? C->kA[p->cell] : C->kA_void;
  p->tauS = -log(u1) / kS;
  p->tauA = -log(u2) / kA;
  if (kS != 1.0) p->w *= orc_path_weight(kS, p->tauS);
  if (kA != 1.0) p->w *= orc_path_weight(kA, p->tauA);
}

/* Scattering (Sect. 2.1): new direction from the HG phase function of the
 * current frequency, azimuth measured from the plane of the radius vector and
 * the old direction; with scattering weighting (Eq. 7) from an HG function
 * of g_S about the reference direction instead, azimuth from the plane of
 * the reference and the old direction.  Both free paths redrawn (Eq. 1). */
static void do_scatter(orc_ctx *C, orc_pkg *p, orc_stream *rs, int s)
{
  double u_mu, u_phi;
  draw2(rs, &u_mu, &u_phi);
  double phi = 2.0 * ORC_PI * u_phi;
  double e1[3], e2[3], dn[3];
  if (C->M->scat_w) {
    double ref[3];
    reference_direction(p, s, ref);
    double mr = orc_hg_mu(C->M->g_S, u_mu);
    double sr = sqrt(fmax(0.0, 1.0 - mr * mr));
    frame(ref, p->d, e1, e2);
    for (int i = 0; i < 3; ++i) dn[i] = mr * ref[i] + sr * (cos(phi) * e1[i] + sin(phi) * e2[i]);
    normalise3(dn);
    double mu_s = dot3(p->d, dn);
    p->w *= orc_hg_pdf2(C->M->g[p->f], mu_s) / orc_hg_pdf2(C->M->g_S, mr);
  } else {
    double mu_s = orc_hg_mu(C->M->g[p->f], u_mu);
    double st = sqrt(fmax(0.0, 1.0 - mu_s * mu_s));
    double xr = sqrt(dot3(p->x, p->x));
    frame(p->d, xr > 0.0 ? p->x : NULL, e1, e2);
    for (int i = 0; i < 3; ++i) dn[i] = mu_s * p->d[i] + st * (cos(phi) * e1[i] + sin(phi) * e2[i]);
    normalise3(dn);
  }
  memcpy(p->d, dn, sizeof dn);
  draw_paths(C, p, rs);
  p->nev[0] += 1;
  C->st[ST_SCATTER] += 1.0;
  record(p, ORC_EV_SCATTER, p->cell, p->f);
}

/* Absorption and immediate re-emission (Sect. 2.1).  Returns 0 when the
 * package ends (terminal frozen mode). */
static int do_absorb(orc_ctx *C, orc_pkg *p, orc_stream *rs, int s)
{
  const orc_model *M = C->M;
  int F = C->F, c = p->cell;
  double dE = p->w * C->eps[s];
  C->st[ST_ABSORB] += 1.0;
  p->nev[1] += 1;
  if (C->mode == ORC_MODE_FROZEN_TERMINAL) {
    C->E[c] += dE;
    record(p, ORC_EV_ABSORB, c, p->f);
    return 0;
  }
  double u_e, u_nu, u_mu, u_phi;
  draw2(rs, &u_e, &u_nu);
  (void)u_e;
  double E_new = C->E[c] + dE;
  C->E[c] = E_new;
  int fn;
  if (C->mode == ORC_MODE_IRE) {
    /* new temperature from the exact energy balance, then the frequency from
     * the difference spectrum kabs [B(T_new) - B(T_old)] dnu */
    double e = E_new / C->mass[c];
    if (e > C->Lmax) C->st[ST_CLAMP_HI] += 1.0;
    double Tn = solve_temperature(F, M->freq, C->dnu, M->kabs, e, C->T[c], C->L_lo, C->L_hi);
    double *Bc = C->Bcur + (size_t)c * F;
    double pdiff[ORC_MAX_FREQ], tot = 0.0;
    for (int k = 0; k < F; ++k) {
      double bn = M->kabs[k] * orc_planck(M->freq[k], Tn) * C->dnu[k];
      pdiff[k] = bn - Bc[k];
      if (pdiff[k] < 0.0) pdiff[k] = 0.0;
      tot += pdiff[k];
      Bc[k] = bn;
    }
    if (!(tot > 0.0)) {
      for (int k = 0; k < F; ++k) pdiff[k] = M->kabs[k] * orc_dplanck_dT(M->freq[k], Tn) * C->dnu[k];
    }
    C->T[c] = Tn;
    double cdf[ORC_MAX_FREQ];
    make_cdf(F, pdiff, cdf);
    fn = sample_cdf(F, cdf, u_nu);
  } else {
    fn = sample_cdf(F, C->cdf_frozen + (size_t)c * F, u_nu);
  }
  p->f = fn;
  if (M->remit_random) {
    double u_r, u_spare;
    draw2(rs, &u_r, &u_spare);
    (void)u_spare;
    double rn = orc_shell_radius(M->radii[c], M->radii[c + 1], u_r);
    double xr = sqrt(dot3(p->x, p->x));
    if (xr > 0.0) {
      for (int i = 0; i < 3; ++i) p->x[i] *= rn / xr;
    } else {
      p->x[0] = 0.0; p->x[1] = 0.0; p->x[2] = rn;
    }
  }
  draw2(rs, &u_mu, &u_phi);
  double phi = 2.0 * ORC_PI * u_phi;
  double e1[3], e2[3];
  if (M->g_E != 0.0) {
    /* weighted re-emission (Eq. 6): HG(g_E) about the reference direction,
     * weight = isotropic density / HG density */
    double ref[3];
    reference_direction(p, s, ref);
    double mr = orc_hg_mu(M->g_E, u_mu);
    double sr = sqrt(fmax(0.0, 1.0 - mr * mr));
    frame(ref, NULL, e1, e2);
    for (int i = 0; i < 3; ++i) p->d[i] = mr * ref[i] + sr * (cos(phi) * e1[i] + sin(phi) * e2[i]);
    p->w /= orc_hg_pdf2(M->g_E, mr);
  } else {
    /* isotropic new direction: mu uniform in [-1,1] about the radius vector */
    double mu = 2.0 * u_mu - 1.0;
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    double rhat[3] = {0.0, 0.0, 1.0};
    double xr = sqrt(dot3(p->x, p->x));
    if (xr > 0.0)
      for (int i = 0; i < 3; ++i) rhat[i] = p->x[i] / xr;
    frame(rhat, NULL, e1, e2);
    for (int i = 0; i < 3; ++i) p->d[i] = mu * rhat[i] + st * (cos(phi) * e1[i] + sin(phi) * e2[i]);
  }
  normalise3(p->d);
  draw_paths(C, p, rs);
  record(p, ORC_EV_ABSORB, c, fn);
  return 1;
}

/* Cross into the next cell; returns 0 when the package has left the model. */
static int do_cross(orc_ctx *C, orc_pkg *p, int next, double l, int s)
{
  move(p, l);
  p->cell = next;
  p->nev[2] += 1;
  C->st[ST_CROSS] += 1.0;
  record(p, ORC_EV_CROSS, next, p->f);
  if (next >= C->n) {
    escape(C, p, s);
    return 0;
  }
  return 1;
}

/* Total extinction optical depth tau0 from the current point to the surface
 * along the current direction (Sect. 2.2.2). */
static double prewalk_tau(const orc_ctx *C, const orc_pkg *p0)
{
  orc_pkg q = *p0;
  double acc = 0.0;
  while (q.cell < C->n) {
    int next;
    double l = boundary_distance(C, q.x, q.d, q.cell, &next);
    acc += (kabs_cell(C, q.cell, q.f) + ksca_cell(C, q.cell, q.f)) * l;
    move(&q, l);
    q.cell = next;
  }
  return acc;
}

/* Absorption and scattering optical depths, summed separately, from the
 * current point to the surface along the current direction. */
static void prewalk_tau_split(const orc_ctx *C, const orc_pkg *p0, double *tauA0, double *tauS0)
{
  orc_pkg q = *p0;
  double a = 0.0, b = 0.0;
  while (q.cell < C->n) {
    int next;
    double l = boundary_distance(C, q.x, q.d, q.cell, &next);
    a += kabs_cell(C, q.cell, q.f) * l;
    b += ksca_cell(C, q.cell, q.f) * l;
    move(&q, l);
    q.cell = next;
  }
  *tauA0 = a;
  *tauS0 = b;
}

static void simulate(orc_ctx *C, int s, uint64_t pkg, uint64_t seed, uint32_t *nev_out, uint64_t *hash_out)
{
  const orc_model *M = C->M;
  orc_stream rs;
  stream_init(&rs, seed, pkg, M->model_id, (uint32_t)s);
  orc_pkg p;
  memset(&p, 0, sizeof p);
  p.hash = FNV_OFFSET;
  p.w = 1.0;

  /* ---- injection (Sect. 2.1, Eqs. 1-3; weighting Eq. 5) */
  double u_f, u_mu;
  draw2(&rs, &u_f, &u_mu);
  p.f = sample_cdf(C->F, C->cdf_src[s], u_f);
  p.cell = (s == 0) ? C->n - 1 : ((M->radii[0] > 0.0) ? -1 : 0);
  double w_path = 1.0;  /* free-path weight of the first flight (Eq. 8) */
  if (M->ffi) {
    double u1, u2;  /* the forced flight replaces these paths */
    draw2(&rs, &u1, &u2);
    p.tauS = -log(u1);
    p.tauA = -log(u2);
  } else {
    draw_paths(C, &p, &rs);
    w_path = p.w;
    p.w = 1.0;
  }
  double mu;
  if (s == 0) {
    if (M->k_bg == 0.5) {
      mu = sqrt(u_mu);
    } else {
      mu = pow(u_mu, M->k_bg);
      p.w = 2.0 * M->k_bg * pow(mu, 2.0 - 1.0 / M->k_bg);
    }
    p.x[0] = 0.0; p.x[1] = 0.0; p.x[2] = -C->R;
  } else {
    mu = 2.0 * u_mu - 1.0;
    p.x[0] = p.x[1] = p.x[2] = 0.0;
  }
  p.d[0] = sqrt(fmax(0.0, 1.0 - mu * mu));
  p.d[1] = 0.0;
  p.d[2] = mu;
  /* the injected energy is the source's: before the free-path weight */
  C->st[ST_INJECTED] += 1.0;
  C->st[ST_E_INJECTED] += p.w * C->eps[s];
  p.w *= w_path;
  record(&p, ORC_EV_INJECT, p.cell, p.f);

  int alive = 1;
  if (p.w < 1e-10) {
    lose(C, &p, s, ST_KILL_WEIGHT);
    alive = 0;
  }

  /* ---- forced first interaction (Sect. 2.2.2, Eqs. 9-12) */
  if (alive && M->ffi == 1) {
    double u_int, u_type;
    draw2(&rs, &u_int, &u_type);
    double tau0 = prewalk_tau(C, &p);
    double q = -expm1(-tau0);            /* 1 - e^-tau0 = weight factor, Eq. 12 */
    double e_direct = p.w * C->eps[s] * (1.0 - q);
    C->sed[p.f] += e_direct;
    C->st[ST_E_DIRECT] += e_direct;
    C->st[ST_E_ESCAPED] += e_direct;
    p.w *= q;
    if (!(q > 0.0)) {
      alive = 0;                          /* nothing to interact with: all escaped directly */
      C->st[ST_ESCAPED] += 1.0;
    } else if (p.w < 1e-10) {
      lose(C, &p, s, ST_KILL_WEIGHT);
      alive = 0;
    } else {
      double tau_int = -log1p(-u_int * q);  /* Eq. 10 */
      if (tau_int > tau0) tau_int = tau0;
      double acc = 0.0;
      C->st[ST_FORCED] += 1.0;
      for (;;) {
        int next;
        double l = boundary_distance(C, p.x, p.d, p.cell, &next);
        double ka = kabs_cell(C, p.cell, p.f), ks = ksca_cell(C, p.cell, p.f), ke = ka + ks;
        if (ke > 0.0 && acc + ke * l >= tau_int) {
          double li = (tau_int - acc) / ke;
          if (li > l) li = l;
          if (li < 0.0) li = 0.0;
          move(&p, li);
          p.events += 1;
          if (u_type * ke < ka) alive = do_absorb(C, &p, &rs, s);
          else do_scatter(C, &p, &rs, s);
          if (alive && p.w < 1e-10) {
            lose(C, &p, s, ST_KILL_WEIGHT);
            alive = 0;
          }
          break;
        }
        acc += ke * l;
        p.events += 1;
        if (!do_cross(C, &p, next, l, s)) { alive = 0; break; }   /* unreachable in exact arithmetic */
      }
    }
  }

  /* ---- forced first absorption (Sect. 2.2.2, the forced interaction on the
   * optical depth of absorption only).  tau_S keeps its plain draw.  If it
   * is at least the scattering depth tau_S0 of the whole first ray (the
   * boundary wins ties), the package leaves the ray unscattered unless it is
   * absorbed: the absorption depth is then drawn from the law conditioned on
   * tau < tau_A0 (Eqs. 9-10 with tau_A0 for tau0), the package carries
   * 1 - e^-tau_A0 (Eq. 12) and the rest escapes directly (tallied).  Else the
   * flight runs unforced, with tau_A = -ln(1 - u_int). */
  if (alive && M->ffi == 2) {
    double u_int, u_unused;
    draw2(&rs, &u_int, &u_unused);
    double tauA0, tauS0;
    prewalk_tau_split(C, &p, &tauA0, &tauS0);
    if (p.tauS >= tauS0) {
      double q = -expm1(-tauA0);
      double e_direct = p.w * C->eps[s] * (1.0 - q);
      C->sed[p.f] += e_direct;
      C->st[ST_E_DIRECT] += e_direct;
      C->st[ST_E_ESCAPED] += e_direct;
      p.w *= q;
      if (!(q > 0.0)) {
        alive = 0;
        C->st[ST_ESCAPED] += 1.0;
      } else if (p.w < 1e-10) {
        lose(C, &p, s, ST_KILL_WEIGHT);
        alive = 0;
      } else {
        double tau_int = -log1p(-u_int * q);
        if (tau_int > tauA0) tau_int = tauA0;
        double acc = 0.0;
        C->st[ST_FORCED] += 1.0;
        for (;;) {
          int next;
          double l = boundary_distance(C, p.x, p.d, p.cell, &next);
          double ka = kabs_cell(C, p.cell, p.f);
          if (ka > 0.0 && acc + ka * l >= tau_int) {
            double li = (tau_int - acc) / ka;
            if (li > l) li = l;
            if (li < 0.0) li = 0.0;
            move(&p, li);
            p.events += 1;
            alive = do_absorb(C, &p, &rs, s);
            if (alive && p.w < 1e-10) {
              lose(C, &p, s, ST_KILL_WEIGHT);
              alive = 0;
            }
            break;
          }
          acc += ka * l;
          p.events += 1;
          if (!do_cross(C, &p, next, l, s)) { alive = 0; break; }   /* unreachable in exact arithmetic */
        }
      }
    } else {
      p.tauA = -log1p(-u_int);
    }
  }

  /* ---- main transport loop (Sect. 2.1, Eq. 4) */
  uint64_t cap = C->max_events;
  while (alive) {
    if (p.events >= cap) {
      lose(C, &p, s, ST_KILL_CAP);
      break;
    }
    int next;
    double l = boundary_distance(C, p.x, p.d, p.cell, &next);
    double ka = kabs_cell(C, p.cell, p.f), ks = ksca_cell(C, p.cell, p.f);
    p.events += 1;
    if (p.tauA >= ka * l && p.tauS >= ks * l) {
      p.tauA -= ka * l;
      p.tauS -= ks * l;
      if (!do_cross(C, &p, next, l, s)) break;
    } else if (ka <= 0.0 || p.tauS * ka < p.tauA * ks) {
      /* tau_S ran out first; with no absorption in the cell (ka = 0, only
       * reachable when tau_A is exactly 0) the interaction is a scattering */
      move(&p, p.tauS / ks);
      do_scatter(C, &p, &rs, s);
    } else {
      move(&p, p.tauA / ka);
      if (!do_absorb(C, &p, &rs, s)) break;
    }
    if (p.w < 1e-10) {
      lose(C, &p, s, ST_KILL_WEIGHT);
      break;
    }
  }
  if (nev_out) { nev_out[0] = p.nev[0]; nev_out[1] = p.nev[1]; nev_out[2] = p.nev[2]; }
  if (hash_out) *hash_out = p.hash;
}

/* Validate the model; 0 = fine, negative = invalid. */
int orc_validate(const orc_model *M)
{
  if (!M || M->n_cells < 1 || M->n_freq < 2 || M->n_freq > ORC_MAX_FREQ) return -1;
  if (!M->radii || !M->rho || !M->freq || !M->kabs || !M->ksca || !M->g) return -1;
  if (!(M->radii[0] >= 0.0)) return -2;
  for (int i = 0; i < M->n_cells; ++i) {
    if (!(M->radii[i + 1] > M->radii[i])) return -2;
    if (!(M->rho[i] >= 0.0) || !isfinite(M->rho[i])) return -3;
  }
  for (int k = 0; k < M->n_freq; ++k) {
    if (!(M->freq[k] > 0.0) || (k > 0 && !(M->freq[k] > M->freq[k - 1]))) return -4;
    if (!(M->kabs[k] >= 0.0) || !(M->ksca[k] >= 0.0) || !(fabs(M->g[k]) < 1.0)) return -5;
  }
  if (!M->J_ext && !(M->L_point > 0.0)) return -6;
  if (M->L_point > 0.0 && !M->point_spec) return -6;
  if (!(M->k_bg > 0.0 && M->k_bg <= 1.0)) return -7;
  if (M->ffi < 0 || M->ffi > 2) return -7;
  if (!(fabs(M->g_E) < 1.0) || !(fabs(M->g_S) < 1.0)) return -7;
  if (!(M->k_A > 0.0 && isfinite(M->k_A)) || !(M->k_S > 0.0 && isfinite(M->k_S))) return -7;
  if (M->kA_rho && !(M->kA_lo > 0.0 && isfinite(M->kA_lo) && M->kA_hi > 0.0 && isfinite(M->kA_hi))) return -7;
  if (!(M->length_unit_cm > 0.0)) return -8;
  return 0;
}

/* Luminosities (erg/s) of the two sources: external L = 4 pi^2 R^2 L_u^2
 * sum_k J_k dnu_k (inward flux pi J through the surface 4 pi R^2); point
 * source L_point as given. */
int orc_source_luminosity(const orc_model *M, double *L_out)
{
  double dnu[ORC_MAX_FREQ];
  if (orc_validate(M) < 0) return -1;
  orc_freq_weights(M->n_freq, M->freq, dnu);
  double R = M->radii[M->n_cells] * M->length_unit_cm;
  L_out[0] = 0.0;
  if (M->J_ext) {
    double s = 0.0;
    for (int k = 0; k < M->n_freq; ++k) s += M->J_ext[k] * dnu[k];
    L_out[0] = 4.0 * ORC_PI * ORC_PI * R * R * s;
  }
  L_out[1] = (M->L_point > 0.0) ? M->L_point : 0.0;
  return 0;
}

/* Emission normalisation of each cell: mass_i = 4 pi rho_i V_i L_u^2 with V_i
 * the shell volume in length units, so that the cell emits mass_i * Lambda(T). */
int orc_cell_mass(const orc_model *M, double *mass)
{
  double Lu2 = M->length_unit_cm * M->length_unit_cm;
  for (int i = 0; i < M->n_cells; ++i) {
    double a = M->radii[i], b = M->radii[i + 1];
    double V = 4.0 * ORC_PI / 3.0 * (b - a) * (b * b + a * b + a * a);
    mass[i] = 4.0 * ORC_PI * M->rho[i] * V * Lu2;
  }
  return 0;
}

/* Absorption free-path weighting factor k_A per cell (Sect. 2.2.2): the
 * constant k_A, or with density dependence linear in log density from k_A_lo
 * at the lowest positive cell density to k_A_hi at the highest; empty cells
 * and the central void take k_A_lo. */
int orc_kA_cells(const orc_model *M, double *kA, double *kA_void)
{
  int n = M->n_cells;
  if (!M->kA_rho) {
    for (int i = 0; i < n; ++i) kA[i] = M->k_A;
    *kA_void = M->k_A;
    return 0;
  }
  double lmin = 0.0, lmax = 0.0;
  int any = 0;
  for (int i = 0; i < n; ++i) {
    if (!(M->rho[i] > 0.0)) continue;
    double l = log(M->rho[i]);
    if (!any || l < lmin) lmin = l;
    if (!any || l > lmax) lmax = l;
    any = 1;
  }
  for (int i = 0; i < n; ++i) {
    if (!(M->rho[i] > 0.0)) kA[i] = M->kA_lo;
    else if (!(lmax > lmin)) kA[i] = M->kA_hi;
    else kA[i] = M->kA_hi + (M->kA_lo - M->kA_hi) * (lmax - log(M->rho[i])) / (lmax - lmin);
  }
  *kA_void = M->kA_lo;
  return 0;
}

/*
 * Run N packages per active source (external first, then point source).
 *   mode      ORC_MODE_IRE, ORC_MODE_FROZEN (temperatures fixed to T_frozen,
 *             re-emission from the full cell spectrum kabs B(T_i) dnu) or
 *             ORC_MODE_FROZEN_TERMINAL (absorption ends the package).
 *   E_abs     [n] absorbed energy per cell (erg/s)
 *   T_out     [n] final temperatures (IRE: exact root, clipped to
 *             [T_min, T_max]; frozen modes: T_frozen)
 *   sed       [F] escaping luminosity per frequency bin (erg/s)
 *   stats     [ST_COUNT]
 *   n_events  [N_total*3] scatter, absorb, cross per package, or NULL
 *   hash      [N_total] FNV-1a path hash per package, or NULL
 * Package j of source s is row s_index*N + j, s_index counting active sources.
 */
int orc_run(const orc_model *M, uint64_t N, uint64_t seed, int mode, const double *T_frozen,
            double *E_abs, double *T_out, double *sed, double *stats, uint32_t *n_events,
            uint64_t *hash)
{
  int rc = orc_validate(M);
  if (rc < 0) return rc;
  if (mode != ORC_MODE_IRE && !T_frozen) return -9;
  orc_ctx C;
  memset(&C, 0, sizeof C);
  C.M = M;
  C.n = M->n_cells;
  C.F = M->n_freq;
  C.R = M->radii[C.n];
  C.mode = mode;
  C.sed = sed;
  C.st = stats;
  C.max_events = M->max_events ? M->max_events : 100000000ULL;
  orc_freq_weights(C.F, M->freq, C.dnu);
  double L[2];
  orc_source_luminosity(M, L);
  double p[ORC_MAX_FREQ];
  C.active[0] = (M->J_ext != NULL);
  C.active[1] = (M->L_point > 0.0);
  if (C.active[0]) {
    for (int k = 0; k < C.F; ++k) p[k] = M->J_ext[k] * C.dnu[k];
    make_cdf(C.F, p, C.cdf_src[0]);
  }
  if (C.active[1]) {
    for (int k = 0; k < C.F; ++k) p[k] = M->point_spec[k] * C.dnu[k];
    make_cdf(C.F, p, C.cdf_src[1]);
  }
  for (int s = 0; s < 2; ++s) C.eps[s] = (N > 0) ? L[s] / (double)N : 0.0;

  int n = C.n, F = C.F;
  C.mass = (double *)calloc((size_t)n, sizeof(double));
  C.E = (double *)calloc((size_t)n, sizeof(double));
  C.T = (double *)calloc((size_t)n, sizeof(double));
  C.Bcur = (double *)calloc((size_t)n * F, sizeof(double));
  C.cdf_frozen = (double *)calloc((size_t)n * F, sizeof(double));
  C.kA = (double *)calloc((size_t)n, sizeof(double));
  if (!C.mass || !C.E || !C.T || !C.Bcur || !C.cdf_frozen || !C.kA) {
    free(C.mass); free(C.E); free(C.T); free(C.Bcur); free(C.cdf_frozen); free(C.kA);
    return -10;
  }
  orc_kA_cells(M, C.kA, &C.kA_void);
  orc_cell_mass(M, C.mass);
  C.Lmax = orc_emission(F, M->freq, C.dnu, M->kabs, M->T_max);
  C.L_lo = orc_emission(F, M->freq, C.dnu, M->kabs, ORC_T_LO);
  C.L_hi = orc_emission(F, M->freq, C.dnu, M->kabs, ORC_T_HI);
  memset(sed, 0, sizeof(double) * F);
  memset(stats, 0, sizeof(double) * ST_COUNT);
  if (mode != ORC_MODE_IRE) {
    for (int i = 0; i < n; ++i) {
      for (int k = 0; k < F; ++k) p[k] = M->kabs[k] * orc_planck(M->freq[k], T_frozen[i]) * C.dnu[k];
      make_cdf(F, p, C.cdf_frozen + (size_t)i * F);
    }
  }
  uint64_t row = 0;
  for (int s = 0; s < 2; ++s) {
    if (!C.active[s]) continue;
    for (uint64_t j = 0; j < N; ++j, ++row) {
      simulate(&C, s, j, seed, n_events ? n_events + 3 * row : NULL, hash ? hash + row : NULL);
    }
  }
  for (int i = 0; i < n; ++i) {
    E_abs[i] = C.E[i];
    if (mode == ORC_MODE_IRE) {
      double T = (C.E[i] > 0.0 && C.mass[i] > 0.0)
                     ? solve_temperature(F, M->freq, C.dnu, M->kabs, C.E[i] / C.mass[i], C.T[i], C.L_lo, C.L_hi)
                     : 0.0;
      if (T < M->T_min) T = M->T_min;
      if (T > M->T_max) T = M->T_max;
      T_out[i] = T;
    } else {
      T_out[i] = T_frozen[i];
    }
  }
  free(C.mass); free(C.E); free(C.T); free(C.Bcur); free(C.cdf_frozen); free(C.kA);
  return 0;
}

int orc_stat_count(void) { return ST_COUNT; }
