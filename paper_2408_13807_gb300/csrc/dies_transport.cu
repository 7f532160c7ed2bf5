// dies_transport.cu -- the IRE transport kernel (Sect. 2.1 with the weighting
// of Sect. 2.2), the temperature kernel and the FP32 batch merge.
//
// Design (GB300): one persistent grid sized to the SM count; every thread
// owns one photon package at a time, its state in registers; a warp refills
// its finished lanes from a device work counter with one atomic per refill
// (ballot + popc), so that lanes keep stepping while long-lived packages of
// the same warp finish.  One loop iteration performs exactly one event per
// live lane (boundary crossing, scattering or absorption + re-emission), so
// the warp stays converged at the loop head.  Per-frequency tables and the
// emission table are staged in shared memory; the re-emission CDF rows and
// the per-cell geometry are read through L1.  Absorbed energies are FP64
// atomics whose returned old value gives the (E_old, E_new) pair of the
// absorption, so every GPU run is one serialisation of the IRE updates.
//
// Geometry is one-dimensional: the impact parameter p^2 is invariant along a
// straight flight and s = r mu is the signed path coordinate, r^2 = p^2 + s^2.
// At each boundary s is set afresh to +-sqrt(R_b^2 - p^2), so no rounding
// accumulates along a flight and precision is relative to the local radius.
#include "dies_common.cuh"

namespace dies {
namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr unsigned kFull = 0xffffffffu;

enum Phase { PH_DEAD = 0, PH_PREWALK = 1, PH_FORCED = 2, PH_NORMAL = 3 };

template <int PREC>
struct RealOf {
  using T = float;
};
template <>
struct RealOf<PREC_FP64> {
  using T = double;
};

// Shared-memory tables of one CTA.
struct Shared {
  float kabs_f[kMaxFreq], ksca_f[kMaxFreq];
  float hg_a[kMaxFreq], hg_b[kMaxFreq], hg_c[kMaxFreq], hg_1pg2[kMaxFreq], hg_inv2g[kMaxFreq];
  float src_cdf_f[2][kMaxFreq];
  double kabs_d[kMaxFreq], ksca_d[kMaxFreq], g_d[kMaxFreq];
  double src_cdf_d[2][kMaxFreq];
  double sed[kMaxFreq];
};

template <class Real>
struct Lane {
  Real p2, s, tauA, tauS, w, acc, tau_int, s0, u_type;
  double eps;
  int cell, f, phase, cell0, src, model, cell_off, bnd, n, n64;
  uint32_t events;
  Stream rs;
  // parity records
  unsigned long long row, hash;
  uint32_t nsca, nabs, ncross;
};

struct Tally {
  uint32_t c[CNT_COUNT];
  double e_inj, e_lost, e_direct;
};

// ------------------------------------------------------------- sampling
// smallest k with cdf[k] >= u over a 64-entry row (entries >= F hold 1)
template <class T>
__device__ __forceinline__ int cdf_pick(const T *row, T u) {
  int k = 0;
#pragma unroll
  for (int step = 32; step > 0; step >>= 1)
    if (row[k + step - 1] < u) k += step;
  return k;
}
__device__ __forceinline__ int cdf_pick_ldg(const float *row, float u) {
  int k = 0;
#pragma unroll
  for (int step = 32; step > 0; step >>= 1)
    if (__ldg(row + k + step - 1) < u) k += step;
  return k;
}
__device__ __forceinline__ int cdf_pick_ldg(const double *row, double u) {
  int k = 0;
#pragma unroll
  for (int step = 32; step > 0; step >>= 1)
    if (__ldg(row + k + step - 1) < u) k += step;
  return k;
}

// number of table nodes with Lambda_j <= e (table padded with +inf to pow2)
__device__ __forceinline__ int node_count_f(const float *L, int pow2, float e) {
  int j = 0;
  for (int step = pow2 >> 1; step > 0; step >>= 1)
    if (L[j + step - 1] <= e) j += step;
  if (L[j] <= e) ++j;  // L[pow2-1] is +inf for a padded table, finite only if n == pow2
  return j;
}

// the exact FP64 count, starting from a float estimate
__device__ __forceinline__ int node_count_d(const double *Ld, int n, int j, double e) {
  while (j < n && __ldg(Ld + j) <= e) ++j;
  while (j > 0 && __ldg(Ld + j - 1) > e) --j;
  return j;
}

// ------------------------------------------------------------ geometry
template <class Real>
__device__ __forceinline__ Real ld_r2(const TransportParams &P, int b);
template <>
__device__ __forceinline__ float ld_r2<float>(const TransportParams &P, int b) {
  return __ldg(P.r2f + b);
}
template <>
__device__ __forceinline__ double ld_r2<double>(const TransportParams &P, int b) {
  return __ldg(P.r2d + b);
}

// Distance l to the boundary through which the package leaves its cell, the
// path coordinate sb of that boundary, and the cell entered there.
template <int PREC, class Real>
__device__ __forceinline__ void boundary(const TransportParams &P, const Lane<Real> &L, Real &l, Real &sb,
                                         int &next) {
  const int c = L.cell;
  const int bi = L.bnd + (c >= 0 ? c : 0);
  const Real lo2 = (c >= 0) ? ld_r2<Real>(P, bi) : Real(0);
  const Real hi2 = ld_r2<Real>(P, bi + (c >= 0 ? 1 : 0));
  const bool inward = (L.s < Real(0)) && (L.p2 < lo2);
  next = inward ? c - 1 : c + 1;
  if constexpr (PREC == PREC_FP64) {
    // cancellation-free forms of the two roots of |x + l d|^2 = R^2
    const Real r2 = L.p2 + L.s * L.s;
    if (inward) {
      const Real sq = sqrt(lo2 - L.p2);
      l = (r2 - lo2) / (-L.s + sq);
      sb = -sq;
    } else {
      const Real sq = sqrt(fmax(hi2 - L.p2, 0.0));
      l = (L.s <= 0.0) ? (-L.s + sq) : ((hi2 - r2) / (L.s + sq));
      sb = sq;
    }
    l = fmax(l, 0.0);
  } else {
    if (PREC == PREC_MIXED && c >= 0 && c < L.n64) {
      // innermost shells: crossing distance in FP64 (R^2 - p^2 cancels there)
      const double t2 = __ldg(P.r2d + bi + (inward ? 0 : 1));
      double sq = sqrt(fmax(t2 - (double)L.p2, 0.0));
      if (inward) sq = -sq;
      sb = (float)sq;
      l = fmaxf((float)(sq - (double)L.s), 0.0f);
    } else {
      float sq = sqrtf(fmaxf((inward ? lo2 : hi2) - L.p2, 0.0f));
      sb = inward ? -sq : sq;
      l = fmaxf(sb - L.s, 0.0f);
    }
  }
}

// ---------------------------------------------------------- bookkeeping
template <bool RECORD, class Real>
__device__ __forceinline__ void record(Lane<Real> &L, int ev, int cell, int f) {
  if constexpr (RECORD) L.hash = fnv_word(L.hash, event_word(ev, cell, f));
}

template <bool RECORD, class Real>
__device__ __forceinline__ void finish(const TransportParams &P, Lane<Real> &L) {
  L.phase = PH_DEAD;
  if constexpr (RECORD) {
    if (P.rec_events) {
      P.rec_events[3 * L.row + 0] = L.nsca;
      P.rec_events[3 * L.row + 1] = L.nabs;
      P.rec_events[3 * L.row + 2] = L.ncross;
    }
    if (P.rec_hash) P.rec_hash[L.row] = L.hash;
  }
}

template <bool RECORD, class Real>
__device__ __forceinline__ void escape(const TransportParams &P, Shared &S, Lane<Real> &L, Tally &T) {
  const double e = (double)L.w * L.eps;
  if (P.n_models == 1) atomicAdd(&S.sed[L.f], e);
  else atomicAdd(P.sed + (size_t)L.model * kMaxFreq + L.f, e);
  T.c[CNT_ESCAPED]++;
  finish<RECORD>(P, L);
}

template <bool RECORD, class Real>
__device__ __forceinline__ void lose(const TransportParams &P, Lane<Real> &L, Tally &T, int why) {
  T.c[why]++;
  T.e_lost += (double)L.w * L.eps;
  finish<RECORD>(P, L);
}

template <bool RECORD, class Real>
__device__ __forceinline__ void cross(const TransportParams &P, Shared &S, Lane<Real> &L, Tally &T, Real sb,
                                      int next) {
  L.s = sb;
  L.cell = next;
  T.c[CNT_CROSS]++;
  if constexpr (RECORD) L.ncross++;
  record<RECORD>(L, EV_CROSS, next, L.f);
  if (next >= L.n) escape<RECORD>(P, S, L, T);
}

// ------------------------------------------------------------ injection
template <int PREC, bool RECORD>
__device__ void inject(const TransportParams &P, Shared &S, Lane<typename RealOf<PREC>::T> &L,
                       unsigned long long g, Tally &T) {
  using Real = typename RealOf<PREC>::T;
  // work index -> (source slot, package); slots are numbered model by model
  const unsigned long long slot = g / P.pkg_len;
  const unsigned long long pkg = P.pkg_begin + (g - slot * P.pkg_len);
  int m = 0;
  if (P.n_models > 1) {
    int lo = 0, hi = P.n_models - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(&P.desc[mid].pkg_off) <= slot) lo = mid; else hi = mid - 1;
    }
    m = lo;
  }
  const ModelDesc *D = P.desc + m;
  const unsigned long long sl = slot - __ldg(&D->pkg_off);
  const int mask = __ldg(&D->src_mask);
  const int src = (mask == 3) ? (int)sl : ((mask & 1) ? 0 : 1);
  L.model = m;
  L.src = src;
  L.cell_off = __ldg(&D->cell_off);
  L.bnd = __ldg(&D->bnd_off);
  L.n = __ldg(&D->n_cells);
  L.n64 = __ldg(&D->n_fp64);
  L.eps = __ldg(&D->L[src]) / (double)P.n_per_source;
  const double R = __ldg(&D->R);
  L.rs.k0 = (uint32_t)P.seed;
  L.rs.k1 = (uint32_t)(P.seed >> 32);
  L.rs.c0 = (uint32_t)pkg;
  L.rs.c1 = (uint32_t)(pkg >> 32);
  L.rs.c3 = (uint32_t)m ^ ((uint32_t)src << 24);
  L.rs.blk = 0;
  L.events = 0;
  L.w = Real(1);
  if constexpr (RECORD) {
    L.row = sl * P.n_per_source + pkg;
    L.hash = 0xcbf29ce484222325ULL;
    L.nsca = L.nabs = L.ncross = 0;
  }
  Real u_int = Real(0.5);
  if constexpr (PREC == PREC_FP64) {
    const U4 a = L.rs.next();
    const double u_f = u01d(a.x, a.y), u_mu = u01d(a.z, a.w);
    L.f = cdf_pick(S.src_cdf_d[src], u_f);
    const U4 b = L.rs.next();
    L.tauS = -log(u01d(b.x, b.y));
    L.tauA = -log(u01d(b.z, b.w));
    if (src == 0) {
      double mu;
      if (P.k_bg == 0.5) {
        mu = sqrt(u_mu);
      } else {
        mu = pow(u_mu, P.k_bg);
        L.w = 2.0 * P.k_bg * pow(mu, 2.0 - 1.0 / P.k_bg);
      }
      L.s = -R * mu;
      L.p2 = R * R - L.s * L.s;
      L.cell = L.n - 1;
    } else {
      L.s = 0.0;
      L.p2 = 0.0;
      L.cell = __ldg(&D->point_cell);
    }
    if (P.ffi) {
      const U4 c = L.rs.next();
      u_int = u01d(c.x, c.y);
      L.u_type = u01d(c.z, c.w);
    }
  } else {
    const U4 a = L.rs.next();
    L.f = cdf_pick(S.src_cdf_f[src], u01f_word(a.x));
    const float v = u01f_fine(a.y);  // 1 - u of the direction draw
    L.tauS = -__logf(u01f_word(a.z));
    L.tauA = -__logf(u01f_word(a.w));
    if (src == 0) {
      const float Rf = (float)R;
      float mu, sin2;
      if (P.k_bg == 0.5) {
        mu = sqrtf(1.0f - v);
        sin2 = v;
      } else {
        // mu = u^k, 1 - mu^2 = -expm1(2k ln u), weight 2k u^(2k-1) (Eq. 5)
        const float k = (float)P.k_bg;
        const float lnu = log1pf(-v);
        mu = expf(k * lnu);
        sin2 = -expm1f(2.0f * k * lnu);
        L.w = 2.0f * k * expf((2.0f * k - 1.0f) * lnu);
      }
      L.s = -Rf * mu;
      L.p2 = Rf * Rf * sin2;
      L.cell = L.n - 1;
    } else {
      L.s = 0.0f;
      L.p2 = 0.0f;
      L.cell = __ldg(&D->point_cell);
    }
    if (P.ffi) {
      const U4 c = L.rs.next();
      u_int = u01f_word(c.x);
      L.u_type = u01f_word(c.y);
    }
  }
  T.c[CNT_INJECTED]++;
  T.e_inj += (double)L.w * L.eps;
  record<RECORD>(L, EV_INJECT, L.cell, L.f);
  if (L.w < Real(1e-10)) {
    lose<RECORD>(P, L, T, CNT_KILL_WEIGHT);
    return;
  }
  if (P.ffi) {
    L.phase = PH_PREWALK;
    L.acc = Real(0);
    L.tau_int = u_int;  // holds u_int until the pre-walk has found tau0
    L.s0 = L.s;
    L.cell0 = L.cell;
  } else {
    L.phase = PH_NORMAL;
  }
}

// ----------------------------------------------------------- scattering
template <int PREC, bool RECORD>
__device__ __forceinline__ void scatter(const TransportParams &P, Shared &S, Lane<typename RealOf<PREC>::T> &L,
                                        Tally &T) {
  if constexpr (PREC == PREC_FP64) {
    const U4 a = L.rs.next();
    const double u_mu = u01d(a.x, a.y), u_phi = u01d(a.z, a.w);
    const double g = S.g_d[L.f];
    double mu_s;
    if (fabs(g) < 1e-6) {
      mu_s = 2.0 * u_mu - 1.0;
    } else {
      const double t = (1.0 - g * g) / (1.0 - g + 2.0 * g * u_mu);
      mu_s = fmin(fmax((1.0 + g * g - t * t) / (2.0 * g), -1.0), 1.0);
    }
    const double st = sqrt(fmax(0.0, 1.0 - mu_s * mu_s));
    const double r2 = L.p2 + L.s * L.s;
    const double r = sqrt(r2);
    if (r > 0.0) {
      const double mu = L.s / r, sth = sqrt(fmax(L.p2, 0.0)) / r;
      const double mup = mu * mu_s + sth * st * cos(kTwoPi * u_phi);
      L.s = r * mup;
      L.p2 = fmax(r2 - L.s * L.s, 0.0);
    } else {
      L.s = 0.0;
      L.p2 = 0.0;
    }
    const U4 b = L.rs.next();
    L.tauS = -log(u01d(b.x, b.y));
    L.tauA = -log(u01d(b.z, b.w));
  } else {
    const U4 a = L.rs.next();
    const float u = u01f_word(a.x), u_phi = u01f_word(a.y);
    const int f = L.f;
    float mu_s, st2;
    const float gb = S.hg_b[f];  // 1 - g
    if (S.hg_c[f] == 0.0f) {
      mu_s = 2.0f * u - 1.0f;
      st2 = 4.0f * u * (1.0f - u);
    } else {
      // HG inversion; 1 - mu_s in a cancellation-free form for forward angles
      const float den = fmaf(S.hg_c[f], u, gb);
      const float t = __fdividef(S.hg_a[f], den);
      mu_s = fminf(fmaxf((S.hg_1pg2[f] - t * t) * S.hg_inv2g[f], -1.0f), 1.0f);
      const float omt = fminf(__fdividef(gb * (1.0f - u) * (t + gb), den), 2.0f);
      st2 = omt * (2.0f - omt);
    }
    const float st = sqrtf(st2);
    const float r2 = L.p2 + L.s * L.s;
    if (r2 > 0.0f) {
      const float rinv = rsqrtf(r2);
      const float r = r2 * rinv;
      const float mu = L.s * rinv, sth = sqrtf(L.p2) * rinv;
      float sp, cp;
      __sincosf(6.2831853f * u_phi, &sp, &cp);
      const float mup = mu * mu_s + sth * st * cp;
      // sin^2 of the new radial angle from |r_hat x d'|^2 (no 1 - mu'^2 cancellation)
      const float q = mu * st * cp - sth * mu_s;
      const float sin2 = st2 * sp * sp + q * q;
      L.s = r * mup;
      L.p2 = r2 * sin2;
    } else {
      L.s = 0.0f;
      L.p2 = 0.0f;
    }
    L.tauS = -__logf(u01f_word(a.z));
    L.tauA = -__logf(u01f_word(a.w));
  }
  T.c[CNT_SCATTER]++;
  if constexpr (RECORD) L.nsca++;
  record<RECORD>(L, EV_SCATTER, L.cell, L.f);
}

// ---------------------------------------------- absorption + re-emission
template <int PREC, int MODE, bool RECORD>
__device__ __forceinline__ void absorb(const TransportParams &P, Shared &S, const float *sLnode,
                                       Lane<typename RealOf<PREC>::T> &L, Tally &T) {
  using Real = typename RealOf<PREC>::T;
  const int gc = L.cell_off + L.cell;
  T.c[CNT_ABSORB]++;
  if constexpr (RECORD) L.nabs++;
  const double dE = (double)L.w * L.eps;
  if constexpr (MODE == MODE_FROZEN_TERMINAL) {
    atomicAdd(P.E + gc, dE);
    record<RECORD>(L, EV_ABSORB, L.cell, L.f);
    finish<RECORD>(P, L);
    return;
  }
  if constexpr (PREC == PREC_FP64) {
    const U4 a = L.rs.next();
    const double u_e = u01d(a.x, a.y), u_nu = u01d(a.z, a.w);
    if constexpr (MODE == MODE_FROZEN) {
      atomicAdd(P.E + gc, dE);
      L.f = cdf_pick_ldg(P.cell_cdf + (size_t)gc * kMaxFreq, u_nu);
    } else {
      const double old = atomicAdd(P.E + gc, dE);
      const double im = __ldg(P.inv_mass + gc);
      const double eo = old * im, en = (old + dE) * im;
      const double es = eo + u_e * (en - eo);
      int j = node_count_f(sLnode, P.n_tnodes_pow2, (float)es);
      j = node_count_d(P.Lnode_d, P.n_tnodes, min(j, P.n_tnodes), es);
      if (en > __ldg(P.Lnode_d + P.n_tnodes - 1)) T.c[CNT_CLAMP_HI]++;
      const int row = min(j, P.n_tnodes - 1);
      L.f = cdf_pick_ldg(P.dcdf_d + ((size_t)row << kFreqShift), u_nu);
    }
    const U4 b = L.rs.next();
    const double mu = 2.0 * u01d(b.x, b.y) - 1.0;
    const double r2 = L.p2 + L.s * L.s;
    const double r = sqrt(r2);
    L.s = r * mu;
    L.p2 = fmax(r2 - L.s * L.s, 0.0);
    const U4 c = L.rs.next();
    L.tauS = -log(u01d(c.x, c.y));
    L.tauA = -log(u01d(c.z, c.w));
  } else {
    // one Philox block gives five 23-bit uniforms (4 x top bits + 1 from the low bits)
    const U4 a = L.rs.next();
    const float u_e = u01f_word(a.x), u_nu = u01f_word(a.y), u_mu = u01f_word(a.z);
    const float u_ts = u01f_word(a.w);
    const float u_ta = u01f((a.x & 0x1ffu) | ((a.y & 0x1ffu) << 9) | ((a.z & 0x1fu) << 18));
    int row;
    if constexpr (PREC == PREC_MIXED) {
      const double old = atomicAdd(P.E + gc, dE);
      const double im = __ldg(P.inv_mass + gc);
      const double eo = old * im, en = (old + dE) * im;
      const double es = eo + (double)u_e * (en - eo);
      int j = node_count_f(sLnode, P.n_tnodes_pow2, (float)es);
      j = node_count_d(P.Lnode_d, P.n_tnodes, min(j, P.n_tnodes), es);
      if (en > __ldg(P.Lnode_d + P.n_tnodes - 1)) T.c[CNT_CLAMP_HI]++;
      row = min(j, P.n_tnodes - 1);
    } else {
      // FP32 form: two FP32 counters, E = E_prev (frozen in this batch) + E_cur
      const float dEf = (float)dE;
      const float oc = atomicAdd(P.Ecur + gc, dEf);
      const float Eo = __ldg(P.Eprev + gc) + oc;
      const float En = Eo + dEf;
      const float im = __ldg(P.inv_massf + gc);
      const float eo = Eo * im, en = En * im;
      const float es = fmaf(u_e, en - eo, eo);
      const int j = node_count_f(sLnode, P.n_tnodes_pow2, es);
      if (en > sLnode[P.n_tnodes - 1]) T.c[CNT_CLAMP_HI]++;
      row = min(j, P.n_tnodes - 1);
    }
    L.f = cdf_pick_ldg(P.dcdf_f + ((size_t)row << kFreqShift), u_nu);
    // isotropic re-emission: mu' = 2u - 1, sin^2 = 4u(1-u)
    const float r2 = L.p2 + L.s * L.s;
    const float r = sqrtf(r2);
    L.s = r * (2.0f * u_mu - 1.0f);
    L.p2 = r2 * (4.0f * u_mu * (1.0f - u_mu));
    L.tauS = -__logf(u_ts);
    L.tauA = -__logf(u_ta);
  }
  record<RECORD>(L, EV_ABSORB, L.cell, L.f);
}

// ------------------------------------------------------------ one event
template <int PREC, int MODE, bool RECORD>
__device__ __forceinline__ void step(const TransportParams &P, Shared &S, const float *sLnode,
                                     Lane<typename RealOf<PREC>::T> &L, Tally &T) {
  using Real = typename RealOf<PREC>::T;
  if (L.phase == PH_NORMAL && L.events >= P.max_events) {
    lose<RECORD>(P, L, T, CNT_KILL_CAP);
    return;
  }
  Real l, sb;
  int next;
  boundary<PREC>(P, L, l, sb, next);
  Real ka = Real(0), ks = Real(0);
  if (L.cell >= 0) {
    if constexpr (PREC == PREC_FP64) {
      const double rho = __ldg(P.rhod + L.cell_off + L.cell);
      ka = S.kabs_d[L.f] * rho;
      ks = S.ksca_d[L.f] * rho;
    } else {
      const float rho = __ldg(P.rhof + L.cell_off + L.cell);
      ka = S.kabs_f[L.f] * rho;
      ks = S.ksca_f[L.f] * rho;
    }
  }
  if (L.phase == PH_PREWALK) {
    // total extinction optical depth to the surface (Sect. 2.2.2)
    L.acc += (ka + ks) * l;
    L.s = sb;
    L.cell = next;
    if (next >= L.n) {
      const Real tau0 = L.acc;
      Real q;
      if constexpr (PREC == PREC_FP64) q = -expm1(-tau0);
      else q = -expm1f(-tau0);
      const double e_direct = (double)L.w * L.eps * (1.0 - (double)q);
      if (P.n_models == 1) atomicAdd(&S.sed[L.f], e_direct);
      else atomicAdd(P.sed + (size_t)L.model * kMaxFreq + L.f, e_direct);
      T.e_direct += e_direct;
      L.w *= q;
      if (!(q > Real(0))) {
        T.c[CNT_ESCAPED]++;
        finish<RECORD>(P, L);
      } else if (L.w < Real(1e-10)) {
        lose<RECORD>(P, L, T, CNT_KILL_WEIGHT);
      } else {
        Real ti;
        if constexpr (PREC == PREC_FP64) ti = -log1p(-L.tau_int * q);  // Eq. 10
        else ti = -log1pf(-L.tau_int * q);
        L.tau_int = (ti > tau0) ? tau0 : ti;
        T.c[CNT_FORCED]++;
        L.s = L.s0;
        L.cell = L.cell0;
        L.acc = Real(0);
        L.phase = PH_FORCED;
      }
    }
    return;
  }
  L.events++;
  if (L.phase == PH_FORCED) {
    const Real ke = ka + ks;
    if (ke > Real(0) && L.acc + ke * l >= L.tau_int) {
      Real li = (L.tau_int - L.acc) / ke;
      li = li > l ? l : li;
      li = li < Real(0) ? Real(0) : li;
      L.s += li;
      L.phase = PH_NORMAL;
      if (L.u_type * ke < ka) absorb<PREC, MODE, RECORD>(P, S, sLnode, L, T);
      else scatter<PREC, RECORD>(P, S, L, T);
    } else {
      L.acc += ke * l;
      cross<RECORD>(P, S, L, T, sb, next);
    }
    return;
  }
  // normal transport: competing free paths (Eqs. 1 and 4); the boundary wins
  // ties, and an interaction in a cell without absorption is a scattering
  const Real ta = ka * l, ts = ks * l;
  if (L.tauA >= ta && L.tauS >= ts) {
    L.tauA -= ta;
    L.tauS -= ts;
    cross<RECORD>(P, S, L, T, sb, next);
  } else if (ka <= Real(0) || L.tauS * ka < L.tauA * ks) {
    L.s += L.tauS / ks;
    scatter<PREC, RECORD>(P, S, L, T);
  } else {
    L.s += L.tauA / ka;
    absorb<PREC, MODE, RECORD>(P, S, sLnode, L, T);
  }
  if (L.phase != PH_DEAD && L.w < Real(1e-10)) lose<RECORD>(P, L, T, CNT_KILL_WEIGHT);
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <int PREC, int MODE, bool RECORD>
__global__ void __launch_bounds__(256) k_transport(const TransportParams P) {
  using Real = typename RealOf<PREC>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Shared &S = *reinterpret_cast<Shared *>(smem_raw);
  float *sLnode = reinterpret_cast<float *>(smem_raw + sizeof(Shared));

  for (int k = threadIdx.x; k < kMaxFreq; k += blockDim.x) {
    const bool in = k < P.F;
    const double ka = in ? P.kabs_d[k] : 0.0, ks = in ? P.ksca_d[k] : 0.0, g = in ? P.g_d[k] : 0.0;
    S.kabs_d[k] = ka;
    S.ksca_d[k] = ks;
    S.g_d[k] = g;
    S.kabs_f[k] = (float)ka;
    S.ksca_f[k] = (float)ks;
    const bool iso = fabs(g) < 1e-6;
    S.hg_a[k] = (float)(1.0 - g * g);
    S.hg_b[k] = (float)(1.0 - g);
    S.hg_c[k] = iso ? 0.0f : (float)(2.0 * g);
    S.hg_1pg2[k] = (float)(1.0 + g * g);
    S.hg_inv2g[k] = iso ? 0.0f : (float)(0.5 / g);
    for (int s = 0; s < 2; ++s) {
      S.src_cdf_d[s][k] = P.src_cdf_d[s * kMaxFreq + k];
      S.src_cdf_f[s][k] = (float)P.src_cdf_d[s * kMaxFreq + k];
    }
    S.sed[k] = 0.0;
  }
  for (int j = threadIdx.x; j < P.n_tnodes_pow2; j += blockDim.x) sLnode[j] = P.Lnode_f[j];
  __syncthreads();

  Tally T;
#pragma unroll
  for (int i = 0; i < CNT_COUNT; ++i) T.c[i] = 0;
  T.e_inj = T.e_lost = T.e_direct = 0.0;

  Lane<Real> L;
  L.phase = PH_DEAD;
  bool exhausted = false;
  const int lane = threadIdx.x & 31;
  const unsigned long long t0 = globaltimer();
  unsigned iter = 0;
  for (;;) {
    const unsigned need = __ballot_sync(kFull, L.phase == PH_DEAD && !exhausted);
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(P.queue, (unsigned long long)__popc(need));
      base = __shfl_sync(kFull, base, leader);
      if (need & (1u << lane)) {
        const unsigned long long g = base + __popc(need & ((1u << lane) - 1u));
        if (g < P.total) inject<PREC, RECORD>(P, S, L, g, T);
        else exhausted = true;
      }
    }
    if (!__any_sync(kFull, L.phase != PH_DEAD)) break;
    if (L.phase != PH_DEAD) step<PREC, MODE, RECORD>(P, S, sLnode, L, T);
    if ((++iter & 1023u) == 0) {
      const bool late = (globaltimer() - t0) > P.time_budget_ns;
      if (__shfl_sync(kFull, late, 0)) {
        if (lane == 0) atomicOr(P.status, STATUS_TIMEOUT);
        break;
      }
    }
  }

  // counters: warp reduction, one atomic per warp
#pragma unroll
  for (int i = 0; i < CNT_COUNT; ++i) {
    unsigned long long v = T.c[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if (lane == 0 && v) atomicAdd(P.counters + i, v);
  }
  double ev[EN_COUNT] = {T.e_inj, T.e_lost, T.e_direct};
#pragma unroll
  for (int i = 0; i < EN_COUNT; ++i) {
    double v = ev[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if (lane == 0 && v != 0.0) atomicAdd(P.energies + i, v);
  }
  __syncthreads();
  if (P.n_models == 1)
    for (int k = threadIdx.x; k < P.F; k += blockDim.x)
      if (S.sed[k] != 0.0) atomicAdd(P.sed + k, S.sed[k]);
}

// Temperature of every cell from its absorbed energy: log-log interpolation
// of T(Lambda) between table nodes; below the first node T_min, above the
// last T_max.
__global__ void k_finalize(int n_cells, const double *E, const float *Eprev, const float *Ecur, int fp32,
                           const double *inv_mass, const double *Lnode, const double *lnT, int n, double *T_out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  const double Ec = fp32 ? (double)(Eprev[c] + Ecur[c]) : E[c];
  const double e = Ec * inv_mass[c];
  double lT;
  if (!(e >= Lnode[0])) {
    lT = lnT[0];
  } else if (e >= Lnode[n - 1]) {
    lT = lnT[n - 1];
  } else {
    int lo = 0, hi = n - 1;  // Lnode[lo] <= e < Lnode[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (Lnode[mid] <= e) lo = mid; else hi = mid;
    }
    const double x = (log(e) - log(Lnode[lo])) / (log(Lnode[hi]) - log(Lnode[lo]));
    lT = lnT[lo] + x * (lnT[hi] - lnT[lo]);
  }
  T_out[c] = exp(lT);
}

// FP32 form, end of a batch: fold the current-batch counter into the
// previous-batches counter (Sect. 2.3).
__global__ void k_merge_batches(int n_cells, float *Eprev, float *Ecur) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n_cells) {
    Eprev[c] += Ecur[c];
    Ecur[c] = 0.0f;
  }
}

template <int PREC, int MODE, bool RECORD>
cudaError_t launch_one(const TransportParams &P, int grid, int block, size_t smem, cudaStream_t st) {
  auto kern = k_transport<PREC, MODE, RECORD>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, block, smem, st>>>(P);
  launch_counter_add(1);
  return cudaGetLastError();
}

template <int PREC, int MODE, bool RECORD>
cudaError_t occupancy_one(int block, size_t smem, int *blocks_per_sm) {
  auto kern = k_transport<PREC, MODE, RECORD>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, block, smem);
}

}  // namespace

size_t transport_smem_bytes(int n_tnodes_pow2) { return sizeof(Shared) + sizeof(float) * (size_t)n_tnodes_pow2; }

// prec: PREC_*, mode: MODE_*; the frozen modes exist in the FP64 form only.
cudaError_t launch_transport(int prec, int mode, bool record, const TransportParams &P, int grid, int block,
                             cudaStream_t st) {
  const size_t smem = transport_smem_bytes(P.n_tnodes_pow2);
  if (mode != MODE_IRE) {
    if (prec != PREC_FP64) return cudaErrorInvalidValue;
    if (mode == MODE_FROZEN)
      return record ? launch_one<PREC_FP64, MODE_FROZEN, true>(P, grid, block, smem, st)
                    : launch_one<PREC_FP64, MODE_FROZEN, false>(P, grid, block, smem, st);
    return record ? launch_one<PREC_FP64, MODE_FROZEN_TERMINAL, true>(P, grid, block, smem, st)
                  : launch_one<PREC_FP64, MODE_FROZEN_TERMINAL, false>(P, grid, block, smem, st);
  }
  switch (prec) {
    case PREC_MIXED: return launch_one<PREC_MIXED, MODE_IRE, false>(P, grid, block, smem, st);
    case PREC_FP32: return launch_one<PREC_FP32, MODE_IRE, false>(P, grid, block, smem, st);
    default: return launch_one<PREC_FP64, MODE_IRE, false>(P, grid, block, smem, st);
  }
}

cudaError_t transport_occupancy(int prec, int mode, int block, int n_tnodes_pow2, int *blocks_per_sm) {
  const size_t smem = transport_smem_bytes(n_tnodes_pow2);
  if (mode != MODE_IRE) return occupancy_one<PREC_FP64, MODE_FROZEN, true>(block, smem, blocks_per_sm);
  switch (prec) {
    case PREC_MIXED: return occupancy_one<PREC_MIXED, MODE_IRE, false>(block, smem, blocks_per_sm);
    case PREC_FP32: return occupancy_one<PREC_FP32, MODE_IRE, false>(block, smem, blocks_per_sm);
    default: return occupancy_one<PREC_FP64, MODE_IRE, false>(block, smem, blocks_per_sm);
  }
}

cudaError_t launch_finalize(cudaStream_t st, int n_cells, const double *E, const float *Eprev, const float *Ecur,
                            int fp32, const double *inv_mass, const double *Lnode, const double *lnT, int n,
                            double *T_out) {
  const int tb = 256;
  k_finalize<<<(n_cells + tb - 1) / tb, tb, 0, st>>>(n_cells, E, Eprev, Ecur, fp32, inv_mass, Lnode, lnT, n, T_out);
  launch_counter_add(1);
  return cudaGetLastError();
}

cudaError_t launch_merge(cudaStream_t st, int n_cells, float *Eprev, float *Ecur) {
  const int tb = 256;
  k_merge_batches<<<(n_cells + tb - 1) / tb, tb, 0, st>>>(n_cells, Eprev, Ecur);
  launch_counter_add(1);
  return cudaGetLastError();
}

}  // namespace dies
