// dies_transport.cu -- the IRE transport kernel (Sect. 2.1 with the weighting
// of Sect. 2.2), the temperature kernel, the tally conversion and the FP32
// batch merge.
//
// Design (GB300): one persistent grid sized to the SM count; every thread
// owns one photon package at a time, its state in registers.  The inner loop
// moves every live lane by boundary crossings (the common event: tens to
// thousands per package against a handful of interactions).  A lane whose
// free path runs out inside its cell, or that needs a new package, parks
// with a pending rare event; the warp leaves the move loop once enough lanes
// wait (or after inner_moves steps) and runs the rare-event path for all
// parked lanes together, so one pass through the Philox, HG-inversion or
// table-search code serves many lanes instead of one.  Finished lanes refill
// from their warp's chunk of work items; lane 0 takes a new chunk from the
// device work counter when it runs out (one atomic per chunk of 32-1024
// packages instead of one per refill).  Per-frequency tables
// and the emission table are staged in shared memory; the per-cell geometry
// is one 16-byte record read through L1.
//
// Geometry is one-dimensional: the impact parameter p^2 is invariant along a
// straight flight and s = r mu is the signed path coordinate, r^2 = p^2 + s^2.
// At each boundary s is set afresh to +-sqrt(R_b^2 - p^2), so no rounding
// accumulates along a flight and precision is relative to the local radius.
// In the FP32 forms R_b^2 is a float pair (hi + lo = the FP64 square), so
// R_b^2 - p^2 is formed as (hi - p^2) + lo without cancellation.
//
// Accounting: the FP64 form (parity) adds energies in FP64 exactly as the
// oracle does.  The FP32 forms keep FP64 only in the absorbed-energy
// accumulators: escaped, injected and directly escaped weights are summed as
// 64-bit integers in units of 2^-24 package energies and converted once, so
// no FP64 instruction runs per event (GB300's FP64 rate is a small fraction of
// its FP32 rate).
#include "dies_common.cuh"

namespace dies {
namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kCheck = 8;  // moves between two early-exit ballots of the move loop (measured best of 2-32)
constexpr int kMaxWarps = 8;  // warps per CTA (block size <= 256)

// Lane states.  0-2: the package moves; 3: it left the cloud, its escape
// is tallied with the warp's rare events; 4-7: parked until the warp runs its
// rare events (7: the forced-interaction pre-walk reached the surface);
// 8: finished, waiting for a new package; 9: no work left.  Everything beyond
// a crossing runs on the rare path, so the per-crossing path stays short and
// free of divergent branches.
enum State {
  ST_NORMAL = 0, ST_PREWALK = 1, ST_FORCED = 2,
  ST_ESCAPE = 3,
  ST_SCATTER = 4, ST_ABSORB = 5, ST_INJECT = 6, ST_FFIEND = 7,
  ST_DEAD = 8, ST_DONE = 9
};

// Compile-time options of the FP32 / MIXED transport kernels.
constexpr int OPT_R64 = 1;    // MIXED: FP64 crossing distances in the innermost shells of some model
constexpr int OPT_NOFFI = 2;  // no forced first interaction: every moving package is in ST_NORMAL
constexpr int OPT_BATCH = 4;  // several models: per-model injection tallies grouped per warp (add_model_q)
constexpr int OPT_CDF = 8;    // MIXED single model: re-emission bin from FP32 CDF rows instead of alias rows
// every weighting option but the centre-directed background neutral: k_S = 1,
// no per-cell k_A, no directional scattering or re-emission weighting, and
// re-emission at the absorption point.  The branches it drops are never taken
// then, so the results are those of the general kernel; dropping their code
// shortens the kernel (measured 0.3-4 % faster, most with forced interaction).
constexpr int OPT_PLAIN = 16;
// single model, FP32 forms without FP64 crossings: the geometry records
// (16-byte record and density per cell and the void) are staged in shared
// memory, and every crossing reads them there instead of through L1
// (measured +4.6 to +7 % on every mixed-form class: shorter shared-memory
// addressing and latency); the host picks it only where the staged records
// do not reduce the CTAs resident per SM
constexpr int OPT_SGEO = 32;
// FP32 forms, launch knob aggregate_atomics: the warp-aggregated absorption
// atomics compiled in (without it the kernel carries no aggregation code:
// measured +0.6 to +1 % on the classes that do not aggregate)
constexpr int OPT_AGG = 64;

template <int PREC>
struct RealOf {
  using T = float;
};
template <>
struct RealOf<PREC_FP64> {
  using T = double;
};

// Shared-memory tables and tallies of one CTA.
struct alignas(16) Shared {  // 16-byte size: staged geometry records follow it
  float kabs_f[kMaxFreq], ksca_f[kMaxFreq];
  float inv_ka_f[kMaxFreq], inv_ks_f[kMaxFreq];  // 1 / coefficient (inf where it is 0)
  float hg_a[kMaxFreq], hg_b[kMaxFreq], hg_c[kMaxFreq], hg_1pg2[kMaxFreq], hg_inv2g[kMaxFreq];
  uint32_t src_alias[2][kMaxFreq];   // FP32 forms: source spectra as alias tables
  uint16_t nguide[kGuide];           // FP32 forms: node-search guide
  int g_b0, g_sh;
  uint32_t key[2];                   // Philox key (the run's seed)
  double kabs_d[kMaxFreq], ksca_d[kMaxFreq], g_d[kMaxFreq];
  double src_cdf_d[2][kMaxFreq];
  // FP32 forms, single model: 64-bit fixed-point tallies kept as 32-bit
  // halves (lo, hi) so that only 32-bit shared-memory atomics are used
  unsigned int sed_lo[2][kMaxFreq], sed_hi[2][kMaxFreq];
  unsigned int inj_lo[2], inj_hi[2], dir_lo[2], dir_hi[2];
  unsigned int rare[CNT_COUNT];            // per-package counters
  // per-warp work cursor [next, end) within the warp's current chunk;
  // read and written by lane 0 of that warp only
  unsigned long long wq_next[kMaxWarps], wq_end[kMaxWarps];
};

// Shared-memory bytes of n staged geometry records (float4 + float density
// each), rounded to 16 so that the node table after them stays aligned.
__host__ __device__ constexpr size_t sgeo_bytes(int n) { return (20 * (size_t)n + 15) & ~(size_t)15; }

// Byte offset of the per-warp package pools (pool variant) in a CTA's
// dynamic shared memory: after the Shared block and the node table.
__host__ __device__ constexpr size_t pool_offset(int n_tnodes_pow2) {
  return (sizeof(Shared) + sizeof(float) * (size_t)n_tnodes_pow2 + 15) & ~(size_t)15;
}

template <class Real>
struct Lane {
  Real p2, s, tauA, tauS, w, acc, tau_int, s0, u_type;
  // FP32 forms: every flight (normal, forced pre-walk, forced) accumulates
  // the column density acc (density x length) and stops at the column lim
  Real lim;
  int next_ev;   // state at lim (ST_SCATTER or ST_ABSORB)
  int exit_st;   // state on leaving the cloud (ST_ESCAPE, or ST_FFIEND for the pre-walk)
  int cinc;      // 1 if the flight's crossings count as crossings (0 in the pre-walk)
  int lo, span;  // FFI forms: the flight leaves when its next cell falls outside [lo, lo + span)
  Real ka, ks;   // absorption / scattering coefficient per unit density at the current frequency
  Real eps;      // package energy (erg/s)
  int cell, f, st, src, model, cell_off, gbase, n, n64;
  uint32_t events, blk, pkg_lo, pkg_hi;
  // parity records
  unsigned long long row, hash;
  uint32_t nsca, nabs, ncross;
};

struct Tally {
  uint32_t cross, scat, abs;
  double e_inj, e_direct;  // FP64 form only
};

template <int PREC>
__device__ __forceinline__ U4 draw(const Shared &S, Lane<typename RealOf<PREC>::T> &L) {
  const U4 r = philox10(L.pkg_lo, L.pkg_hi, L.blk, (uint32_t)L.model ^ ((uint32_t)L.src << 24), S.key[0], S.key[1]);
  ++L.blk;
  return r;
}

// Fixed-point units of a package weight (w * 2^24): a 32-bit conversion when
// it fits, else the exact integer value of the float from its bits (x >= 2^31
// is an integer; weights stay far below 2^40).
__device__ __forceinline__ unsigned long long quanta(float w) {
  const float x = w * kQuantum;
  if (x < 4.0e9f) return (unsigned long long)__float2uint_rn(x);
  const uint32_t b = __float_as_uint(x);
  const uint32_t sh = min((b >> 23) - 150u, 40u);
  return (unsigned long long)((b & 0x7fffffu) | 0x800000u) << sh;
}

// Exact float -> double and truncating double -> float for non-negative
// finite values, on the integer pipes: GB300 runs FP64 instructions, the
// conversions included, at a small fraction of its FP32 rate.  Zero and
// values below the float normal range map to zero.
__device__ __forceinline__ double f2d_nonneg(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t hi = (b >> 23) ? (b >> 3) + (896u << 20) : 0u;  // exponent bias 127 -> 1023
  return __hiloint2double((int)hi, hi ? (int)(b << 29) : 0);
}
__device__ __forceinline__ float d2f_nonneg(double d) {
  const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
  const uint32_t e = hi >> 20;
  if (e <= 896u) return 0.0f;
  if (e >= 1151u) return __int_as_float(0x7f800000);
  return __uint_as_float(((hi - (896u << 20)) << 3) | (lo >> 29));
}

// ------------------------------------------------------------- sampling
// smallest k with row[k] >= u over a 64-entry row (entries >= F hold 1)
template <class T>
__device__ __forceinline__ int cdf_pick(const T *row, T u) {
  int k = 0;
#pragma unroll
  for (int step = 32; step > 0; step >>= 1)
    if (row[k + step - 1] < u) k += step;
  return k;
}
template <class T>
__device__ __forceinline__ int cdf_pick_ldg(const T *row, T u) {
  int k = 0;
#pragma unroll
  for (int step = 32; step > 0; step >>= 1)
    if (__ldg(row + k + step - 1) < u) k += step;
  return k;
}

// FP32 forms: bin drawn from an alias table row by the 23-bit uniform m
// (top 6 bits: the slot; the other 17: the acceptance test).
__device__ __forceinline__ int alias_pick(const uint32_t *row, uint32_t m23) {
  const uint32_t e = row[m23 >> 17];
  return ((m23 & 0x1ffffu) << 9) < (e >> 6) ? (int)(m23 >> 17) : (int)(e & 63u);
}
__device__ __forceinline__ int alias_pick_ldg(const uint32_t *row, uint32_t m23) {
  const uint32_t e = __ldg(row + (m23 >> 17));
  return ((m23 & 0x1ffffu) << 9) < (e >> 6) ? (int)(m23 >> 17) : (int)(e & 63u);
}

// FP32 forms: number of nodes with Lambda_j <= e (e >= 0) from the guide
// bucket of e and a short forward scan.
__device__ __forceinline__ int node_count_guided(const Shared &S, const float *L, int n, float e) {
  const int d = __float_as_int(e) - S.g_b0;
  const int b = d < 0 ? 0 : min(d >> S.g_sh, kGuide - 1);
  int j = S.nguide[b];
  while (j < n && L[j] <= e) ++j;
  return j;
}
// The same count, also returning the first node above e (+inf past the
// table).  The scan is bounded by n: e itself may be +inf (an energy beyond
// the float range), which every node and the +inf padding would satisfy.
__device__ __forceinline__ int node_count_guided_hi(const Shared &S, const float *L, int n, float e, float &hi) {
  const int d = __float_as_int(e) - S.g_b0;
  const int b = d < 0 ? 0 : min(d >> S.g_sh, kGuide - 1);
  int j = S.nguide[b];
  while (j < n && L[j] <= e) ++j;
  hi = (j < n) ? L[j] : __int_as_float(0x7f800000);
  return j;
}

// ------------------------------------------- weighted sampling (Sect. 2.2)
// Henyey-Greenstein cosine by inversion of its CDF (Eq. 6 form; |g| < 1e-6
// is isotropic) and twice its density, (1 - g^2) / (1 + g^2 - 2 g mu)^(3/2).
__device__ __forceinline__ double hg_mu_d(double g, double u) {
  if (fabs(g) < 1e-6) return 2.0 * u - 1.0;
  const double t = (1.0 - g * g) / (1.0 - g + 2.0 * g * u);
  return fmin(fmax((1.0 + g * g - t * t) / (2.0 * g), -1.0), 1.0);
}
__device__ __forceinline__ double hg_pdf2_d(double g, double mu) {
  const double q = 1.0 + g * g - 2.0 * g * mu;
  return (1.0 - g * g) / (q * sqrt(q));
}
// FP32: the cosine and 1 - cosine^2 (cancellation-free for forward angles)
__device__ __forceinline__ void hg_draw_f(float g, float u, float &mu, float &st2) {
  if (fabsf(g) < 1e-6f) {
    mu = 2.0f * u - 1.0f;
    st2 = 4.0f * u * (1.0f - u);
    return;
  }
  const float b = 1.0f - g, den = fmaf(2.0f * g, u, b);
  const float t = __fdividef(1.0f - g * g, den);
  mu = fminf(fmaxf((1.0f + g * g - t * t) * __fdividef(0.5f, g), -1.0f), 1.0f);
  const float omt = fminf(__fdividef(b * (1.0f - u) * (t + b), den), 2.0f);
  st2 = omt * (2.0f - omt);
}
__device__ __forceinline__ float hg_pdf2_f(float g, float mu) {
  const float q = fmaf(-2.0f * g, mu, 1.0f + g * g);
  return (1.0f - g * g) * rsqrtf(q) / q;
}

// number of table nodes with Lambda_j <= e (table padded with +inf to pow2)
__device__ __forceinline__ int node_count_f(const float *L, int pow2, float e) {
  int j = 0;
  for (int step = pow2 >> 1; step > 0; step >>= 1)
    if (L[j + step - 1] <= e) j += step;
  if (L[j] <= e) ++j;
  return j;
}

// the exact FP64 count, starting from a float estimate
__device__ __forceinline__ int node_count_d(const double *Ld, int n, int j, double e) {
  while (j < n && __ldg(Ld + j) <= e) ++j;
  while (j > 0 && __ldg(Ld + j - 1) > e) --j;
  return j;
}

// The same exact count for e >= 0 with the comparisons on the integer pipes:
// non-negative finite doubles order like their bit patterns.  The float
// estimate j (from the float table) is at most one node off, because adjacent
// nodes differ by far more than a float's rounding.
__device__ __forceinline__ int node_count_bits(const double *Ld, int n, int j, double e) {
  const long long eb = __double_as_longlong(e);
  if (j < n && __double_as_longlong(__ldg(Ld + j)) <= eb) return j + 1;
  if (j > 0 && __double_as_longlong(__ldg(Ld + j - 1)) > eb) return j - 1;
  return j;
}

// ---------------------------------------------------------- bookkeeping
template <bool RECORD, class Real>
__device__ __forceinline__ void record(Lane<Real> &L, int ev, int cell, int f) {
  if constexpr (RECORD) L.hash = fnv_word(L.hash, event_word(ev, cell, f));
}

template <bool RECORD, class Real>
__device__ __forceinline__ void finish(const TransportParams &P, Lane<Real> &L) {
  L.st = ST_DEAD;
  if constexpr (RECORD) {
    if (P.rec_events) {
      P.rec_events[3 * L.row + 0] = L.nsca;
      P.rec_events[3 * L.row + 1] = L.nabs;
      P.rec_events[3 * L.row + 2] = L.ncross;
    }
    if (P.rec_hash) P.rec_hash[L.row] = L.hash;
  }
}

// 64-bit add into a (lo, hi) pair of 32-bit shared-memory words: the carry of
// each add is detected from the value its own atomic returned.  (64-bit
// shared-memory atomics, emulated in software, broke warp convergence in
// divergent code here; 32-bit ones are native.)
__device__ __forceinline__ void smem_add64(unsigned int *lo, unsigned int *hi, unsigned long long q) {
  const unsigned int ql = (unsigned int)q, qh = (unsigned int)(q >> 32);
  const unsigned int old = atomicAdd(lo, ql);
  const unsigned int up = qh + ((old + ql < old) ? 1u : 0u);
  if (up) atomicAdd(hi, up);
}

// Batches: add q to the per-(model, source) counter base[key].  With GROUP
// the lanes of the warp that share the key add with one atomic (a warp's
// lanes mostly carry packages of one model, and every injection of a model
// would otherwise hit the same address: measured 2x on the 4096-model study).
template <bool GROUP>
__device__ __forceinline__ void add_model_q(unsigned long long *base, unsigned key, unsigned long long q) {
  if constexpr (GROUP) {
    const unsigned am = __activemask();
    const unsigned grp = __match_any_sync(am, key);
    unsigned long long tot = 0;
    for (unsigned rest = grp; rest != 0u; rest &= rest - 1u) tot += __shfl_sync(grp, q, __ffs(rest) - 1);
    if ((int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(base + key, tot);
  } else {
    atomicAdd(base + key, q);
  }
}

// add weight w of the current package to an escaping-SED bin
template <int PREC>
__device__ __forceinline__ void tally_sed(const TransportParams &P, Shared &S, Lane<typename RealOf<PREC>::T> &L,
                                          typename RealOf<PREC>::T w) {
  DIES_BOUND(P, L.f >= 0 && L.f < kMaxFreq && L.model >= 0 && L.model < P.n_models, STATUS_BAD_FREQ,
             { L.f = 0; L.model = 0; });
  if constexpr (PREC == PREC_FP64) {
    atomicAdd(P.sed + (size_t)L.model * kMaxFreq + L.f, w * L.eps);  // native FP64 reduction in L2
  } else {
    const unsigned long long q = quanta(w);
    if (P.n_models == 1) smem_add64(&S.sed_lo[L.src][L.f], &S.sed_hi[L.src][L.f], q);
    else atomicAdd(P.sed_q + (((size_t)(blockIdx.x & (P.rep - 1)) * P.n_models + L.model) * 2 + L.src) * kMaxFreq + L.f,
                   q);
  }
}

template <int PREC, bool RECORD>
__device__ __forceinline__ void escape(const TransportParams &P, Shared &S, Lane<typename RealOf<PREC>::T> &L) {
  tally_sed<PREC>(P, S, L, L.w);
  atomicAdd(&S.rare[CNT_ESCAPED], 1u);
  finish<RECORD>(P, L);
}

template <bool RECORD, class Real>
__device__ __forceinline__ void lose(const TransportParams &P, Shared &S, Lane<Real> &L, int why) {
  atomicAdd(&S.rare[why], 1u);
  atomicAdd(P.energies + EN_LOST, (double)L.w * (double)L.eps);  // rare
  finish<RECORD>(P, L);
}

// FP32 forms: the reciprocal square root and the base-2 logarithm as the PTX
// approximate instructions with denormal inputs flushed.  Every argument they
// get is a normal number (d >= 1e-36 in boundary, uniforms >= 2^-24), for
// which the flush changes nothing; it only spares the denormal handling
// around the special-function instruction.
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// -ln u of a uniform u in (0, 1), the free path of Eq. 1 (ln u = ln 2 log2 u)
__device__ __forceinline__ float neg_ln_u(float u) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(u));
  return y * -0.69314718f;
}

// ------------------------------------------------------------ geometry
// Distance l to the boundary through which the package leaves its cell, the
// path coordinate sb of that boundary, the cell entered there, and the
// density of the current cell.
template <int PREC, int OPT>
__device__ __forceinline__ void boundary(const TransportParams &P, const Lane<typename RealOf<PREC>::T> &L,
                                         typename RealOf<PREC>::T &l, typename RealOf<PREC>::T &sb, int &next,
                                         typename RealOf<PREC>::T &rho) {
  int c = L.cell;
  DIES_BOUND(P, c >= -1 && c < L.n, STATUS_BAD_CELL, c = -1);
  if constexpr (PREC == PREC_FP64) {
    // cancellation-free forms of the two roots of |x + l d|^2 = R^2 (as the oracle)
    const int bi = L.cell_off + L.model + (c >= 0 ? c : 0);
    const double lo2 = (c >= 0) ? __ldg(P.r2d + bi) : 0.0;
    const double hi2 = __ldg(P.r2d + bi + (c >= 0 ? 1 : 0));
    rho = (c >= 0) ? __ldg(P.rhod + L.cell_off + c) : 0.0;
    const bool inward = (L.s < 0.0) && (L.p2 < lo2);
    next = inward ? c - 1 : c + 1;
    const double r2 = L.p2 + L.s * L.s;
    if (inward) {
      const double sq = sqrt(lo2 - L.p2);
      l = (r2 - lo2) / (-L.s + sq);
      sb = -sq;
    } else {
      const double sq = sqrt(fmax(hi2 - L.p2, 0.0));
      l = (L.s <= 0.0) ? (-L.s + sq) : ((hi2 - r2) / (L.s + sq));
      sb = sq;
    }
    l = fmax(l, 0.0);
  } else {
    const int gi = L.gbase + c;
    float4 G;
    if constexpr ((OPT & OPT_SGEO) != 0) {
      // records [0, sgeo_n) of the single model after the Shared block, then their densities
      extern __shared__ __align__(16) unsigned char smem_raw[];
      const float4 *sg = reinterpret_cast<const float4 *>(smem_raw + sizeof(Shared));
      G = sg[gi];
      rho = reinterpret_cast<const float *>(sg + P.sgeo_n)[gi];
    } else {
      G = __ldg(P.geo + gi);
      rho = __ldg(P.rhoe + gi);
    }
    const float d_in = (G.x - L.p2) + G.y;
    const bool inward = (L.s < 0.0f) & (d_in > 0.0f);
    // sqrt from the hardware reciprocal square root (relative error ~1e-7),
    // signed on the way; a non-positive d (rounding at a tangent) counts as 1e-36
    const float d = fmaxf(inward ? d_in : (G.z - L.p2) + G.w, 1.0e-36f);
    next = inward ? c - 1 : c + 1;
    sb = (inward ? -d : d) * rsqrt_ftz(d);
    if constexpr ((OPT & OPT_R64) != 0) {
      if ((unsigned)c < (unsigned)L.n64) {
        // optional FP64 crossing distance in the innermost shells
        const double t2 = __ldg(P.r2d + L.gbase - 1 + c + (inward ? 0 : 1));
        const float sq = (float)sqrt(fmax(t2 - (double)L.p2, 0.0));
        sb = inward ? -sq : sq;
      }
    }
    // sb - s >= 0 up to rounding; a step negative by rounding is harmless
    // (the column decreases by a rounding amount, the crossing stands)
    l = sb - L.s;
  }
}

template <int PREC, bool RECORD>
__device__ __forceinline__ void cross(const TransportParams &P, Shared &S, Lane<typename RealOf<PREC>::T> &L,
                                      Tally &T, typename RealOf<PREC>::T sb, int next) {
  L.s = sb;
  L.cell = next;
  T.cross++;
  if constexpr (RECORD) L.ncross++;
  record<RECORD>(L, EV_CROSS, next, L.f);
  if (next >= L.n) L.st = ST_ESCAPE;
}

template <int PREC>
__device__ __forceinline__ void set_freq(const Shared &S, Lane<typename RealOf<PREC>::T> &L, int f) {
  L.f = f;
  if constexpr (PREC == PREC_FP64) {
    L.ka = S.kabs_d[f];
    L.ks = S.ksca_d[f];
  } else {
    L.ka = S.kabs_f[f];
    L.ks = S.ksca_f[f];
  }
}

// FP32 forms: the two free paths tau_S, tau_A (Eqs. 1 and 4) become the
// column densities tau_S / k_S and tau_A / k_A.  Both are reached by the
// same column travelled, so only the smaller and which path it belongs to are
// carried: one multiply-add-compare per crossing.  Interactions without
// absorption and ties resolve as in the FP64 form.
// With free-path weighting (Eq. 8) tau = -ln(u) / k and the package weight
// gains e^(tau (k - 1)) / k per path; the factor is returned (k_A is that of
// the package's current cell).  PLAIN: no free-path weighting (factor 1).
template <bool PLAIN>
__device__ __forceinline__ float set_paths(const TransportParams &P, const Shared &S, Lane<float> &L, float tS,
                                           float tA) {
  float wf = 1.0f;
  if (!PLAIN && P.k_S_f != 1.0f) {
    const float k = P.k_S_f;
    tS = __fdividef(tS, k);
    wf *= __fdividef(__expf(tS * (k - 1.0f)), k);
  }
  if (!PLAIN && P.kA_f) {
    const float k = (L.cell >= 0) ? __ldg(P.kA_f + L.cell_off + L.cell) : P.kA_void_f;
    if (k != 1.0f) {
      tA = __fdividef(tA, k);
      wf *= __fdividef(__expf(tA * (k - 1.0f)), k);
    }
  }
  const float nA = tA * S.inv_ka_f[L.f], nS = tS * S.inv_ks_f[L.f];
  L.acc = 0.0f;
  L.lim = fminf(nA, nS);
  L.next_ev = (nS < nA) ? ST_SCATTER : ST_ABSORB;
  return wf;
}

// FP64 form: both free paths from one block, weighted as the oracle does
// (scattering path first); returns the weight factor.
__device__ __forceinline__ double paths_d(const TransportParams &P, Lane<double> &L, const U4 &b) {
  const double kS = P.k_S;
  const double kA = P.kA_d ? ((L.cell >= 0) ? __ldg(P.kA_d + L.cell_off + L.cell) : P.kA_void) : 1.0;
  L.tauS = -log(u01d(b.x, b.y)) / kS;
  L.tauA = -log(u01d(b.z, b.w)) / kA;
  double wf = 1.0;
  if (kS != 1.0) wf *= exp(L.tauS * (kS - 1.0)) / kS;
  if (kA != 1.0) wf *= exp(L.tauA * (kA - 1.0)) / kA;
  return wf;
}

// ----------------------------------- forced first interaction (Sect. 2.2.2)
// PREWALK accumulates the extinction optical depth tau0 to the surface along
// the first flight; FORCED replays the flight and stops where the cumulative
// extinction reaches tau_int (Eq. 10), choosing absorption with probability
// k_A / k_ext.  Forcing on the absorption depth (P.ffi == 2): the pre-walk
// sums tau_A0 in acc and tau_S0 in u_type, and the forced flight runs on the
// absorption depth alone and always absorbs.  (FP64 form; the FP32 forms run
// both as ordinary flights of the common move, see move.)
template <int PREC, int MODE, bool RECORD>
__device__ __forceinline__ void move_forced(const TransportParams &P, Shared &S, Lane<double> &L, Tally &T) {
  using Real = double;
  Real l, sb, rho;
  int next;
  boundary<PREC, 0>(P, L, l, sb, next, rho);
  const Real ka = L.ka * rho, ks = L.ks * rho;
  if (L.st == ST_PREWALK) {
    if (P.ffi == 2) {
      L.acc += ka * l;
      L.u_type += ks * l;
    } else {
      L.acc += (ka + ks) * l;
    }
    L.s = sb;
    L.cell = next;
    if (next >= L.n) L.st = ST_FFIEND;
    return;
  }
  if constexpr (PREC == PREC_FP64) L.events++;
  const Real ke = (P.ffi == 2) ? ka : ka + ks;
  if (ke > Real(0) && L.acc + ke * l >= L.tau_int) {
    Real li = (L.tau_int - L.acc) / ke;
    li = li > l ? l : li;
    li = li < Real(0) ? Real(0) : li;
    L.s += li;
    L.st = (P.ffi == 2 || L.u_type * ke < ka) ? ST_ABSORB : ST_SCATTER;
  } else {
    L.acc += ke * l;
    cross<PREC, RECORD>(P, S, L, T, sb, next);
  }
}

// -------------------------------------------------- the common event: move
// One step of a moving package: cross into the next cell, or stop at an
// interaction point and park for a scattering / absorption.
//
// FP32 forms: the normal flight, the forced-interaction pre-walk and the
// forced flight are one instruction stream (no divergence between lanes in
// different kinds of flight): accumulate the column x = rho l; stop inside
// the cell where acc + x passes lim (x > 0 there, so rho > 0), else cross.
// The pre-walk has lim = inf and leaves the cloud into ST_FFIEND.
// CALLER_COUNTS: the caller counts crossings per block of moves (FP32 forms)
template <int PREC, int MODE, bool RECORD, int OPT, bool CALLER_COUNTS = false>
__device__ __forceinline__ void move(const TransportParams &P, Shared &S, Lane<typename RealOf<PREC>::T> &L,
                                     Tally &T) {
  using Real = typename RealOf<PREC>::T;
  if constexpr (PREC != PREC_FP64) {
    float l, sb, rho;
    int next;
    boundary<PREC, OPT>(P, L, l, sb, next, rho);
    const float a2 = fmaf(rho, l, L.acc);
    if (a2 > L.lim) {
      L.s += fminf(__fdividef(L.lim - L.acc, rho), l);
      L.st = L.next_ev;
    } else {
      L.acc = a2;
      L.s = sb;
      L.cell = next;
      if constexpr ((OPT & OPT_NOFFI) != 0) {
        if constexpr (!CALLER_COUNTS) T.cross++;
        if (next >= L.n) L.st = ST_ESCAPE;
      } else {
        if constexpr (!CALLER_COUNTS) T.cross += L.cinc;
        if ((unsigned)(next - L.lo) >= (unsigned)L.span) L.st = L.exit_st;
      }
    }
    return;
  } else {
    if (L.st != ST_NORMAL) {
      move_forced<PREC, MODE, RECORD>(P, S, L, T);
      return;
    }
  }
  if constexpr (PREC == PREC_FP64) {
    if (L.events >= P.max_events) {
      lose<RECORD>(P, S, L, CNT_KILL_CAP);
      return;
    }
    L.events++;
  }
  Real l, sb, rho;
  int next;
  boundary<PREC, false>(P, L, l, sb, next, rho);
  const Real ka = L.ka * rho, ks = L.ks * rho;
  // competing free paths (Eqs. 1 and 4); the boundary wins ties, and an
  // interaction in a cell without absorption is a scattering
  const Real ta = ka * l, ts = ks * l;
  if (L.tauA >= ta && L.tauS >= ts) {
    L.tauA -= ta;
    L.tauS -= ts;
    cross<PREC, RECORD>(P, S, L, T, sb, next);
  } else if (ka <= Real(0) || L.tauS * ka < L.tauA * ks) {
    L.s += L.tauS / ks;
    L.st = ST_SCATTER;
  } else {
    L.s += L.tauA / ka;
    L.st = ST_ABSORB;
  }
}

// ------------------------------------------------------------ injection
// Decode work index g into (model, source, package) and reset the lane.
template <int PREC, bool RECORD>
__device__ __forceinline__ void assign(const TransportParams &P, Lane<typename RealOf<PREC>::T> &L,
                                       unsigned long long g) {
  // source slot of work item g (a single model has at most two)
  const unsigned long long slot = (P.n_models == 1) ? (g >= P.pkg_len ? 1ull : 0ull) : g / P.pkg_len;
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
  DIES_BOUND(P, m >= 0 && m < P.n_models, STATUS_BAD_ROW, m = 0);
  const ModelDesc *D = P.desc + m;
  const unsigned long long sl = slot - __ldg(&D->pkg_off);
  const int mask = __ldg(&D->src_mask);
  L.src = (mask == 3) ? (int)sl : ((mask & 1) ? 0 : 1);
  L.model = m;
  L.cell_off = __ldg(&D->cell_off);
  L.gbase = L.cell_off + m + 1;  // geometry record of cell c: gbase + c (void at gbase - 1)
  L.n = __ldg(&D->n_cells);
  L.n64 = __ldg(&D->n_fp64);
  if constexpr (PREC == PREC_FP64) L.eps = __ldg(&D->L[L.src]) / (double)P.n_per_source;
  // FP32 forms: the package energy L / N in float, from two factors scaled
  // by 2^-64 and 2^64 so that a luminosity above the float range (3.4e38)
  // still gives a finite energy
  else L.eps = __ldg(&D->Lf[L.src]) * P.inv_n;  // (2^-64 L)(2^64 / N): finite for any L below 6e57 erg/s
  L.pkg_lo = (uint32_t)pkg;
  L.pkg_hi = (uint32_t)(pkg >> 32);
  L.blk = 0;
  L.events = 0;
  L.st = ST_INJECT;
  if constexpr (RECORD) {
    L.row = sl * P.n_per_source + pkg;
    L.hash = 0xcbf29ce484222325ULL;
    L.nsca = L.nabs = L.ncross = 0;
  }
}

// FP32 forms: the shell holding the turning point r = p of the current
// straight path (the largest boundary b with R_b^2 <= p^2; -1: the central
// void), by bisection over the model's boundary squares.
__device__ __forceinline__ int turning_shell(const TransportParams &P, const Lane<float> &L) {
  const float *R2 = P.r2f + (L.cell_off + L.model);
  if (L.p2 < __ldg(R2)) return -1;
  int lo = 0, hi = L.n;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(R2 + mid) <= L.p2) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Start the package: frequency from the source CDF, free paths (Eq. 1),
// direction (Eqs. 2-3, or Eq. 5 with weighting), optional forced first
// interaction set-up.
template <int PREC, bool RECORD, bool GROUP, bool PLAIN>
__device__ __forceinline__ void inject(const TransportParams &P, Shared &S, Lane<typename RealOf<PREC>::T> &L,
                                       Tally &T, const U4 &a) {
  using Real = typename RealOf<PREC>::T;
  const ModelDesc *D = P.desc + L.model;
  L.w = Real(1);
  Real u_int = Real(0.5);
  Real w_path = Real(1);  // free-path weight of the first flight (Eq. 8), applied after the injection tally
  if constexpr (PREC == PREC_FP64) {
    const double u_f = u01d(a.x, a.y), u_mu = u01d(a.z, a.w);
    int f0 = cdf_pick(S.src_cdf_d[L.src], u_f);
    DIES_BOUND(P, f0 >= 0 && f0 < P.F, STATUS_BAD_FREQ, f0 = 0);
    set_freq<PREC>(S, L, f0);
    const U4 b = draw<PREC>(S, L);
    L.cell = (L.src == 0) ? L.n - 1 : __ldg(&D->point_cell);
    if (P.ffi) {  // the forced flight replaces these paths
      L.tauS = -log(u01d(b.x, b.y));
      L.tauA = -log(u01d(b.z, b.w));
    } else {
      w_path = paths_d(P, L, b);
    }
    if (L.src == 0) {
      const double R = __ldg(&D->R);
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
      const U4 c = draw<PREC>(S, L);
      u_int = u01d(c.x, c.y);
      L.u_type = (P.ffi == 2) ? 0.0 : u01d(c.z, c.w);  // forcing on tau_A: the pre-walk sums tau_S0 here
    }
  } else {
    int f0 = alias_pick(S.src_alias[L.src], a.x >> 9);
    DIES_BOUND(P, f0 >= 0 && f0 < P.F, STATUS_BAD_FREQ, f0 = 0);
    set_freq<PREC>(S, L, f0);
    const float v = u01f_fine(a.y);  // 1 - u of the direction draw
    L.cell = (L.src == 0) ? L.n - 1 : __ldg(&D->point_cell);
    w_path = set_paths<PLAIN>(P, S, L, neg_ln_u(u01f_word(a.z)), neg_ln_u(u01f_word(a.w)));
    if (P.ffi) w_path = 1.0f;  // the forced flight replaces these paths
    if (L.src == 0) {
      const float Rf = __ldg(&D->Rf);
      float mu, sin2;
      if (P.kbg_plain) {
        mu = sqrtf(1.0f - v);
        sin2 = v;
      } else {
        // mu = u^k, 1 - mu^2 = -expm1(2k ln u), weight 2k u^(2k-1) (Eq. 5)
        const float k = P.k_bg_f;
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
      const U4 c = draw<PREC>(S, L);
      u_int = u01f_word(c.x);
      // forcing on tau_A: u_type holds the column to the plain scattering point
      L.u_type = (P.ffi == 2) ? neg_ln_u(u01f_word(a.z)) * S.inv_ks_f[L.f] : u01f_word(c.y);
    }
  }
  atomicAdd(&S.rare[CNT_INJECTED], 1u);
  if constexpr (PREC == PREC_FP64) {
    T.e_inj += (double)L.w * L.eps;
  } else {
    const unsigned long long q = quanta(L.w);
    if (P.n_models == 1) smem_add64(&S.inj_lo[L.src], &S.inj_hi[L.src], q);
    else add_model_q<GROUP>(P.inj_q + (size_t)(blockIdx.x & (P.rep - 1)) * P.n_models * 2,
                            (unsigned)L.model * 2u + (unsigned)L.src, q);
  }
  record<RECORD>(L, EV_INJECT, L.cell, L.f);
  L.w *= w_path;
  if (L.w < Real(1e-10)) {
    lose<RECORD>(P, S, L, CNT_KILL_WEIGHT);
    return;
  }
  if constexpr (PREC != PREC_FP64) {
    L.exit_st = ST_ESCAPE;
    L.cinc = 1;
  }
  if (P.ffi) {
    L.st = ST_PREWALK;
    L.acc = Real(0);
    L.tau_int = u_int;  // holds u_int until the pre-walk has found tau0
    L.s0 = L.s;
    if constexpr (PREC != PREC_FP64) {
      L.lim = __int_as_float(0x7f800000);  // the pre-walk never interacts
      L.exit_st = ST_FFIEND;
      L.cinc = 0;
      L.lo = -1;
      L.span = L.n + 1;  // point source: the radial path to the surface
      L.next_ev = 0;     // 1: mirrored pre-walk
      if (L.src == 0) {
        // An external package's straight path is symmetric about its
        // turning point r = p, so the pre-walk stops on entering the shell
        // that holds the turning point and doubles the column (Sect. 2.2.2
        // needs only the total tau0).
        const int turn = turning_shell(P, L);
        if (turn >= L.n - 1) {
          // the whole chord, 2 R mu, lies in the outermost shell
          L.acc = 2.0f * __ldg(P.rhoe + L.gbase + L.n - 1) * (-L.s);
          L.st = ST_FFIEND;
        } else {
          L.lo = turn + 1;
          L.span = L.n - turn - 1;
          L.next_ev = 1;
        }
      }
    }
  } else {
    L.st = ST_NORMAL;
  }
}

// ----------------------------------------------------------- scattering
template <int PREC, bool RECORD, bool PLAIN>
__device__ __forceinline__ void scatter(const TransportParams &P, Shared &S, Lane<typename RealOf<PREC>::T> &L,
                                        Tally &T, const U4 &a) {
  if constexpr (PREC == PREC_FP64) {
    const double u_mu = u01d(a.x, a.y), u_phi = u01d(a.z, a.w);
    const double g = S.g_d[L.f];
    const double r2 = L.p2 + L.s * L.s;
    const double r = sqrt(r2);
    if (P.scat_w) {
      // Eq. 7: cosine mr to the reference direction (sg r_hat) from HG(g_S),
      // azimuth about it from the plane of the reference and the old direction
      const double sg = (L.src == 0) ? -1.0 : 1.0;
      const double dref = (r > 0.0) ? sg * L.s / r : 1.0;
      const double mr = hg_mu_d(P.g_S, u_mu), sr = sqrt(fmax(0.0, 1.0 - mr * mr));
      const double cos_t = dref * mr + sqrt(fmax(0.0, 1.0 - dref * dref)) * sr * cos(kTwoPi * u_phi);
      L.w *= hg_pdf2_d(g, cos_t) / hg_pdf2_d(P.g_S, mr);
      L.s = r * (sg * mr);
      L.p2 = fmax(r2 - L.s * L.s, 0.0);
    } else {
      const double mu_s = hg_mu_d(g, u_mu);
      const double st = sqrt(fmax(0.0, 1.0 - mu_s * mu_s));
      if (r > 0.0) {
        const double mu = L.s / r, sth = sqrt(fmax(L.p2, 0.0)) / r;
        const double mup = mu * mu_s + sth * st * cos(kTwoPi * u_phi);
        L.s = r * mup;
        L.p2 = fmax(r2 - L.s * L.s, 0.0);
      } else {
        L.s = 0.0;
        L.p2 = 0.0;
      }
    }
    const U4 b = draw<PREC>(S, L);
    L.w *= paths_d(P, L, b);
  } else if (!PLAIN && P.scat_w) {
    // Eq. 7 in FP32: cosine to the reference direction from HG(g_S)
    const float u = u01f_word(a.x), u_phi = u01f_word(a.y);
    const float sg = (L.src == 0) ? -1.0f : 1.0f;
    const float r2 = L.p2 + L.s * L.s;
    float mr, sr2;
    hg_draw_f(P.g_S_f, u, mr, sr2);
    if (r2 > 0.0f) {
      const float rinv = rsqrtf(r2);
      const float dref = sg * L.s * rinv, sth = sqrtf(L.p2) * rinv;  // sth = sin of the old radial angle
      const float cos_t = fminf(fmaxf(fmaf(dref, mr, sth * sqrtf(sr2) * __cosf(6.2831853f * u_phi)), -1.0f), 1.0f);
      L.w *= __fdividef(hg_pdf2_f(S.hg_c[L.f] * 0.5f, cos_t), hg_pdf2_f(P.g_S_f, mr));
      L.s = r2 * rinv * (sg * mr);
      L.p2 = r2 * sr2;
    } else {
      // at r = 0 the reference direction is taken along the old one
      L.w *= __fdividef(hg_pdf2_f(S.hg_c[L.f] * 0.5f, mr), hg_pdf2_f(P.g_S_f, mr));
      L.s = 0.0f;
      L.p2 = 0.0f;
    }
    L.w *= set_paths<PLAIN>(P, S, L, neg_ln_u(u01f_word(a.z)), neg_ln_u(u01f_word(a.w)));
  } else {
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
      L.s = r * mup;
      L.p2 = r2 * (st2 * sp * sp + q * q);
    } else {
      L.s = 0.0f;
      L.p2 = 0.0f;
    }
    L.w *= set_paths<PLAIN>(P, S, L, neg_ln_u(u01f_word(a.z)), neg_ln_u(u01f_word(a.w)));
  }
  T.scat++;
  if constexpr (RECORD) L.nsca++;
  record<RECORD>(L, EV_SCATTER, L.cell, L.f);
}

// Mixed form: the node count of e* = (E_old + u_e dE) / mass formed in FP64
// and searched exactly against the FP64 nodes (E_old = old_d plus the
// energies pre of the lane's aggregation-group predecessors).  Kept out of
// line: inlined, this rarely taken FP64 code slowed the whole kernel by up
// to 9 % (register allocation of the move loop, measured).
__device__ __noinline__ int exact_row(const TransportParams &P, const Shared &S, const float *sLnode, double old_d,
                                      float pre, float u_e, float dEf, int gc) {
  const double od = old_d + f2d_nonneg(pre);
  const double es_d = fma(f2d_nonneg(u_e), f2d_nonneg(dEf), od) * __ldg(P.inv_mass + gc);
  return node_count_bits(P.Lnode_d, P.n_tnodes, node_count_guided(S, sLnode, P.n_tnodes, d2f_nonneg(es_d)), es_d);
}

// ---------------------------------------------- absorption + re-emission
template <int PREC, int MODE, bool RECORD, int OPT>
__device__ __forceinline__ void absorb(const TransportParams &P, Shared &S, const float *sLnode,
                                       Lane<typename RealOf<PREC>::T> &L, Tally &T, const U4 &a) {
  DIES_BOUND(P, L.cell >= 0 && L.cell < L.n, STATUS_BAD_CELL, L.cell = 0);
  const int gc = L.cell_off + L.cell;
  T.abs++;
  if constexpr (RECORD) L.nabs++;
  if constexpr (MODE == MODE_FROZEN_TERMINAL) {
    // the package energy in FP64 in every form (a test mode: the tally must
    // match the FP64 injected energy, not the float package energy)
    if constexpr (PREC == PREC_FP64) atomicAdd(P.E + (size_t)gc * P.e_stride, L.w * L.eps);
    else atomicAdd(P.E + (size_t)gc * P.e_stride, (double)L.w * (__ldg(&P.desc[L.model].L[L.src]) * P.inv_nd));
    record<RECORD>(L, EV_ABSORB, L.cell, L.f);
    finish<RECORD>(P, L);
    return;
  }
  if constexpr (PREC == PREC_FP64) {
    const double dE = L.w * L.eps;
    const double u_e = u01d(a.x, a.y), u_nu = u01d(a.z, a.w);
    int f;
    if constexpr (MODE == MODE_FROZEN) {
      atomicAdd(P.E + (size_t)gc * P.e_stride, dE);
      f = cdf_pick_ldg(P.cell_cdf + (size_t)gc * kMaxFreq, u_nu);
    } else {
      const double old = atomicAdd(P.E + (size_t)gc * P.e_stride, dE);
      const double im = __ldg(P.inv_mass + gc);
      const double eo = old * im, en = (old + dE) * im;
      const double es = eo + u_e * (en - eo);
      int j = node_count_f(sLnode, P.n_tnodes_pow2, (float)es);
      j = node_count_d(P.Lnode_d, P.n_tnodes, min(j, P.n_tnodes), es);
      if (en > __ldg(P.Lnode_d + P.n_tnodes - 1)) atomicAdd(&S.rare[CNT_CLAMP_HI], 1u);
      int row = min(j, P.n_tnodes - 1);
      DIES_BOUND(P, row >= 0, STATUS_BAD_ROW, row = 0);
      f = cdf_pick_ldg(P.dcdf_d + ((size_t)row << kFreqShift), u_nu);
    }
    DIES_BOUND(P, f >= 0 && f < P.F, STATUS_BAD_FREQ, f = 0);
    set_freq<PREC>(S, L, f);
    double rn = -1.0;  // re-emission radius; < 0: the absorption point
    if (P.remit_random) {
      // a point uniform over the cell's volume (the test variant of Sect. 4)
      const U4 e = draw<PREC>(S, L);
      const int bi = L.cell_off + L.model + L.cell;
      const double ri = __ldg(P.radii_d + bi), ro = __ldg(P.radii_d + bi + 1);
      const double a3 = ri * ri * ri;
      rn = cbrt(a3 + u01d(e.x, e.y) * (ro * ro * ro - a3));
    }
    const U4 b = draw<PREC>(S, L);
    double mu;
    if (P.g_E != 0.0) {
      // Eq. 6: cosine to the reference direction from HG(g_E), weight
      // isotropic density / HG density
      const double mr = hg_mu_d(P.g_E, u01d(b.x, b.y));
      mu = (L.src == 0) ? -mr : mr;
      L.w /= hg_pdf2_d(P.g_E, mr);
    } else {
      mu = 2.0 * u01d(b.x, b.y) - 1.0;
    }
    const double r2 = (rn >= 0.0) ? rn * rn : L.p2 + L.s * L.s;
    const double r = (rn >= 0.0) ? rn : sqrt(r2);
    L.s = r * mu;
    L.p2 = fmax(r2 - L.s * L.s, 0.0);
    const U4 c = draw<PREC>(S, L);
    L.w *= paths_d(P, L, c);
  } else {
    // one Philox block gives five 23-bit uniforms (4 x top bits + 1 from the low bits)
    const float u_e = u01f_word(a.x), u_mu = u01f_word(a.z);  // a.y: the re-emission bin
    const float u_ts = u01f_word(a.w);
    const float u_ta = u01f((a.x & 0x1ffu) | ((a.y & 0x1ffu) << 9) | ((a.z & 0x1fu) << 18));
    const float dEf = L.w * L.eps;
    // E_old: MIXED from the FP64 accumulator (old_d, plus pre_d of this lane's
    // group predecessors), as a float in old_f; FP32 form from its two counters
    double old_d = 0.0;
    float old_f = 0.0f, pre_lane = 0.0f;
    if constexpr ((OPT & OPT_AGG) != 0) {
      // Lanes of this warp absorbing in the same cell add their energies
      // with one atomic; each lane's E_old is the group's old value plus the
      // energies of the group's lower lanes (the order of a serial run).
      const unsigned am = __activemask();
      const unsigned grp = __match_any_sync(am, gc);
      const int lane = threadIdx.x & 31, lead = __ffs(grp) - 1;
      const unsigned below = grp & ((1u << lane) - 1u);
      float pre = 0.0f, tot = 0.0f;
      for (unsigned rest = grp; rest != 0u; rest &= rest - 1u) {
        const int j = __ffs(rest) - 1;
        const float v = __shfl_sync(grp, dEf, j);
        tot += v;
        if (below & (1u << j)) pre += v;
      }
      if constexpr (PREC == PREC_MIXED) {
        double old = 0.0;
        if (lane == lead) old = atomicAdd(P.E + (size_t)gc * P.e_stride, f2d_nonneg(tot));
        old_d = __shfl_sync(grp, old, lead);
        old_f = d2f_nonneg(old_d) + pre;
        pre_lane = pre;
      } else {
        float old = 0.0f;
        if (lane == lead) old = __ldg(P.Eprev + gc) + atomicAdd(P.Ecur + (size_t)gc * P.c_stride, tot);
        old_f = __shfl_sync(grp, old, lead) + pre;
      }
    } else if constexpr (PREC == PREC_MIXED) {
      old_d = atomicAdd(P.E + (size_t)gc * P.e_stride, f2d_nonneg(dEf));
      old_f = d2f_nonneg(old_d);
    } else {
      // FP32 form: two FP32 counters, E = E_prev (frozen in this batch) + E_cur
      old_f = __ldg(P.Eprev + gc) + atomicAdd(P.Ecur + (size_t)gc * P.c_stride, dEf);
    }
    if constexpr (PREC == PREC_FP32) {
      if (!(old_f < 1.0e38f)) atomicOr(P.status, STATUS_RANGE);  // the run then reports DIES_ERANGE
    }
    int j;
    float en;  // e_new (table units), for the clamp counter
    if constexpr (PREC == PREC_MIXED) {
      // The row is the node interval holding e* = (E_old + u_e dE) / mass.
      // When e_new stays below the node above e_old by more than float
      // rounding (2^-20 relative), the interval of e_old holds e* for every
      // u_e, and the float energies decide it.  Otherwise (an absorption whose
      // [e_old, e_new] reaches a node: ~1e-4 of them in a well-filled cell)
      // e* is formed in FP64 and searched exactly against the FP64 nodes: in
      // a cell holding more than ~2^24 package energies dE is below one float
      // ulp of E_old, where an FP32 e* would always take the interval of e_old.
      // (the float path also needs the float 1/mass to be a normal number: a
      // very massive cell, e.g. a length unit of ~100 pc, underflows it)
      const float im = __ldg(P.inv_massf + gc);
      const float eo = old_f * im;
      en = fmaf(dEf, im, eo);
      float hi;
      j = node_count_guided_hi(S, sLnode, P.n_tnodes, eo, hi);
      if (!(en < hi * (1.0f - 0x1p-20f)) || !(im >= 0x1p-126f))
        j = exact_row(P, S, sLnode, old_d, pre_lane, u_e, dEf, gc);
    } else {
      const float im = __ldg(P.inv_massf + gc);
      if (!(im >= 0x1p-126f)) atomicOr(P.status, STATUS_RANGE);  // 1/mass below the float range
      const float eo = old_f * im, de = dEf * im;
      j = node_count_guided(S, sLnode, P.n_tnodes, fmaf(u_e, de, eo));
      en = eo + de;
    }
    if (en > sLnode[P.n_tnodes - 1]) atomicAdd(&S.rare[CNT_CLAMP_HI], 1u);
    int row = min(j, P.n_tnodes - 1);
    DIES_BOUND(P, row >= 0, STATUS_BAD_ROW, row = 0);
    // re-emission bin from the row of the interval holding e*: one probe of an
    // alias row, or (kernel variant OPT_CDF) a binary search of an FP32 CDF row
    int f_new;
    if constexpr ((OPT & OPT_CDF) != 0) f_new = cdf_pick_ldg(P.dcdf_f + ((size_t)row << kFreqShift), u01f_word(a.y));
    else f_new = alias_pick_ldg(P.dalias + ((size_t)row << kFreqShift), a.y >> 9);
    int f_chk = f_new;
    DIES_BOUND(P, f_chk >= 0 && f_chk < P.F, STATUS_BAD_FREQ, f_chk = 0);
    set_freq<PREC>(S, L, f_chk);
    float r2 = L.p2 + L.s * L.s;
    float r = sqrtf(r2);
    constexpr bool kPlain = (OPT & OPT_PLAIN) != 0;
    if (!kPlain && P.remit_random) {
      // a point uniform over the cell's volume (the test variant of Sect. 4)
      const U4 e = draw<PREC>(S, L);
      const int bi = L.cell_off + L.model + L.cell;
      const float ri2 = __ldg(P.r2f + bi), ro2 = __ldg(P.r2f + bi + 1);
      const float a3 = ri2 * sqrtf(ri2);
      r = cbrtf(fmaf(u01f_word(e.x), ro2 * sqrtf(ro2) - a3, a3));
      r2 = r * r;
    }
    if (!kPlain && P.g_E_f != 0.0f) {
      // Eq. 6: cosine to the reference direction from HG(g_E)
      float mr, sr2;
      hg_draw_f(P.g_E_f, u_mu, mr, sr2);
      L.s = r * ((L.src == 0) ? -mr : mr);
      L.p2 = r2 * sr2;
      L.w *= __fdividef(1.0f, hg_pdf2_f(P.g_E_f, mr));
    } else {
      // isotropic re-emission: mu' = 2u - 1, sin^2 = 4u(1-u)
      L.s = r * (2.0f * u_mu - 1.0f);
      L.p2 = r2 * (4.0f * u_mu * (1.0f - u_mu));
    }
    L.w *= set_paths<kPlain>(P, S, L, neg_ln_u(u_ts), neg_ln_u(u_ta));
  }
  record<RECORD>(L, EV_ABSORB, L.cell, L.f);
}

// End of the forced-interaction pre-walk: tally the direct escape e^-tau0,
// weight the rest by 1 - e^-tau0 (Eq. 12), draw the forced optical depth
// (Eq. 10) and restart the first flight from the injection point.
//
// Forcing on the absorption depth (P.ffi == 2): only a package whose plain
// scattering clock outlasts the whole first ray is forced, on tau_A0, and it
// always absorbs; any other package restarts an unforced first flight with
// tau_A = -ln(1 - u_int) (an exact split of the analog law given tau_S).
template <int PREC, bool RECORD, bool GROUP>
__device__ __forceinline__ void ffi_end(const TransportParams &P, Shared &S, Lane<typename RealOf<PREC>::T> &L,
                                        Tally &T) {
  using Real = typename RealOf<PREC>::T;
  const bool on_abs = (P.ffi == 2);
  const Real ke = on_abs ? L.ka : L.ka + L.ks;  // per unit density: the coefficient of the forced depth
  Real col0 = L.acc, col_half = Real(0);
  bool mirror = false;
  if constexpr (PREC != PREC_FP64) {
    // a mirrored pre-walk stopped on entering the turning shell (at s <= 0):
    // column to the turning point = acc + rho (0 - s); the path's total twice that
    mirror = (L.next_ev == 1) && L.cell < L.n;  // the turning shell may be the void (-1, density 0)
    if (mirror) {
      col_half = fmaf(__ldg(P.rhoe + L.gbase + L.cell), -L.s, L.acc);
      col0 = 2.0f * col_half;
    } else if (L.next_ev == 1) {
      col0 = L.acc;  // rounding carried it through the turning shell: acc is the whole path
    }
  }
  bool forced = true;
  if (on_abs) {
    if constexpr (PREC == PREC_FP64) forced = (L.tauS >= L.u_type);  // u_type: tau_S0 of the ray
    else forced = !(L.u_type < col0);                                 // u_type: column to the scattering point
  }
  if (!forced) {
    if constexpr (PREC == PREC_FP64) {
      L.tauA = -log1p(-L.tau_int);
    } else {
      const float cA = -log1pf(-L.tau_int) * S.inv_ka_f[L.f];
      L.lim = fminf(cA, L.u_type);
      L.next_ev = (L.u_type < cA) ? ST_SCATTER : ST_ABSORB;
      L.exit_st = ST_ESCAPE;
      L.cinc = 1;
      L.lo = -1;
      L.span = L.n + 1;
    }
    if (mirror && L.lim > col_half) {
      L.s = Real(0);
      L.acc = col_half;
    } else {
      L.s = L.s0;
      L.cell = (L.src == 0) ? L.n - 1 : __ldg(&P.desc[L.model].point_cell);
      L.acc = Real(0);
    }
    L.st = ST_NORMAL;
    return;
  }
  const Real tau0 = (PREC == PREC_FP64) ? L.acc : col0 * ke;
  Real q;
  if constexpr (PREC == PREC_FP64) q = -expm1(-tau0);
  else q = -expm1f(-tau0);
  tally_sed<PREC>(P, S, L, L.w * (Real(1) - q));
  if constexpr (PREC == PREC_FP64) {
    T.e_direct += (double)L.w * L.eps * (1.0 - (double)q);
  } else {
    const unsigned long long dq = quanta(L.w * (1.0f - q));
    if (P.n_models == 1) smem_add64(&S.dir_lo[L.src], &S.dir_hi[L.src], dq);
    else add_model_q<GROUP>(P.dir_q + (size_t)(blockIdx.x & (P.rep - 1)) * P.n_models * 2,
                            (unsigned)L.model * 2u + (unsigned)L.src, dq);
  }
  L.w *= q;
  if (!(q > Real(0))) {
    atomicAdd(&S.rare[CNT_ESCAPED], 1u);
    finish<RECORD>(P, L);
  } else if (L.w < Real(1e-10)) {
    lose<RECORD>(P, S, L, CNT_KILL_WEIGHT);
  } else {
    Real ti;
    if constexpr (PREC == PREC_FP64) {
      ti = -log1p(-L.tau_int * q);  // Eq. 10
      L.tau_int = (ti > tau0) ? tau0 : ti;
    } else {
      // the forced depth as a column (ke > 0 since q > 0); kept strictly
      // below the pre-walk's column, which the replay reproduces exactly
      // (the replay re-walks the path in FP32; the limit stays just short of
      // the pre-walk's total so that the forced interaction happens)
      ti = -log1pf(-L.tau_int * q);
      L.lim = fminf(__fdividef(ti, ke), col0 * (mirror ? 0.99998474f : 0.99999905f));
      L.next_ev = (on_abs || L.u_type * ke < L.ka) ? ST_ABSORB : ST_SCATTER;
      L.exit_st = ST_ESCAPE;
      L.cinc = 1;
      L.lo = -1;
      L.span = L.n + 1;
    }
    atomicAdd(&S.rare[CNT_FORCED], 1u);
    if (mirror && L.lim > col_half) {
      // the forced point lies on the outbound half: replay from the turning point
      L.s = Real(0);
      L.acc = col_half;
    } else if (mirror && L.lim > Real(0.5) * col_half) {
      // the forced point lies on the inbound half, nearer the turning point
      // than the entry: the path is symmetric about the turning point, so
      // walk the mirror image of the stretch from the point to the turning
      // point (outbound from the turning point, to the column
      // col_half - lim) and reflect s at the interaction (s0 = +inf marks
      // it; s0 is not needed once the forced flight has started).  Fewer
      // crossings than a replay from the entry: measured +2 % on forced runs
      L.lim = col_half - L.lim;
      L.s = Real(0);
      L.acc = Real(0);
      if constexpr (PREC != PREC_FP64) L.s0 = __int_as_float(0x7f800000);
    } else {
      L.s = L.s0;
      L.cell = (L.src == 0) ? L.n - 1 : __ldg(&P.desc[L.model].point_cell);
      L.acc = Real(0);
    }
    L.st = ST_FORCED;
  }
}

// The rare-event path for one parked lane.
template <int PREC, int MODE, bool RECORD, int OPT>
__device__ __forceinline__ void rare(const TransportParams &P, Shared &S, const float *sLnode,
                                     Lane<typename RealOf<PREC>::T> &L, Tally &T) {
  constexpr bool kGroup = (OPT & OPT_BATCH) != 0;
  const int kind = L.st;
  // (kernels without forced interaction never reach ST_FFIEND: compiling
  // ffi_end out of them shortens them, measured +1 to +2.7 %)
  if constexpr ((OPT & OPT_NOFFI) == 0) {
    if (kind == ST_FFIEND) {
      ffi_end<PREC, RECORD, kGroup>(P, S, L, T);
      return;
    }
  }
  if constexpr (PREC != PREC_FP64) {
    // the FP32 forms interrupt a package only here, so the event cap is checked here
    if (kind != ST_INJECT && ++L.events >= P.max_events) {
      lose<RECORD>(P, S, L, CNT_KILL_CAP);
      return;
    }
  }
  const U4 a = draw<PREC>(S, L);  // every rare event starts with one Philox block
  L.st = ST_NORMAL;
  if constexpr (PREC != PREC_FP64 && (OPT & OPT_NOFFI) == 0) {
    if (kind != ST_INJECT && L.s0 == __int_as_float(0x7f800000)) {
      L.s = -L.s;  // a forced point reached on the mirrored stretch: back to the inbound half
      L.s0 = 0.0f;
    }
  }
  constexpr bool kPlain = (OPT & OPT_PLAIN) != 0;
  if (kind == ST_INJECT) inject<PREC, RECORD, kGroup, kPlain>(P, S, L, T, a);
  else if (kind == ST_SCATTER) scatter<PREC, RECORD, kPlain>(P, S, L, T, a);
  else absorb<PREC, MODE, RECORD, OPT>(P, S, sLnode, L, T, a);
  // weighted directions and free paths (Eqs. 6-8) change the weight at events:
  // the floor of Sect. 2.2.1 applies after each
  if (kind != ST_INJECT && L.st == ST_NORMAL && L.w < 1e-10f) lose<RECORD>(P, S, L, CNT_KILL_WEIGHT);
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Refill the finished lanes (ST_DEAD) of the warp from the warp's chunk of
// work items: a full-warp collective in which lane 0 alone touches the
// warp's cursor and takes a new chunk from the device counter when this one
// runs out.  A lane beyond the launch's work ends in ST_DONE.
template <int PREC, bool RECORD>
__device__ __forceinline__ void refill(const TransportParams &P, Shared &S, Lane<typename RealOf<PREC>::T> &L) {
  const int lane = threadIdx.x & 31;
  const unsigned dead = __ballot_sync(kFull, L.st == ST_DEAD);
  if (dead == 0u) return;
  const unsigned c = __popc(dead);
  unsigned long long b1 = 0, b2 = 0;
  unsigned n1 = 0;
  if (lane == 0) {
    // P.chunk >= 32 >= c, so one new chunk always covers the shortfall
    const int w = threadIdx.x >> 5;
    const unsigned long long nx = S.wq_next[w];
    n1 = (unsigned)min((unsigned long long)c, S.wq_end[w] - nx);
    b1 = nx;
    if (n1 < c) {
      b2 = atomicAdd(P.queue, (unsigned long long)P.chunk);
      S.wq_next[w] = b2 + (c - n1);
      S.wq_end[w] = b2 + P.chunk;
    } else {
      S.wq_next[w] = nx + n1;
    }
  }
  b1 = __shfl_sync(kFull, b1, 0);
  b2 = __shfl_sync(kFull, b2, 0);
  n1 = __shfl_sync(kFull, n1, 0);
  if (L.st == ST_DEAD) {
    const unsigned r = __popc(dead & ((1u << lane) - 1u));
    const unsigned long long g = (r < n1) ? b1 + r : b2 + (r - n1);
    if (g < P.total) assign<PREC, RECORD>(P, L, g);
    else L.st = ST_DONE;
  }
}

// Per-CTA set-up shared by the transport kernels: per-frequency coefficients,
// HG constants, source tables and the node table into shared memory, tallies
// and work cursors zeroed, the Philox key read (the caller synchronises).
__device__ __forceinline__ void stage_tables(const TransportParams &P, Shared &S, float *sLnode) {
  for (int k = threadIdx.x; k < kMaxFreq; k += blockDim.x) {
    const bool in = k < P.F;
    const double ka = in ? P.kabs_d[k] : 0.0, ks = in ? P.ksca_d[k] : 0.0, g = in ? P.g_d[k] : 0.0;
    S.kabs_d[k] = ka;
    S.ksca_d[k] = ks;
    S.g_d[k] = g;
    S.kabs_f[k] = (float)ka;
    S.ksca_f[k] = (float)ks;
    S.inv_ka_f[k] = (float)(1.0 / ka);  // inf where ka = 0
    S.inv_ks_f[k] = (float)(1.0 / ks);
    const bool iso = fabs(g) < 1e-6;
    S.hg_a[k] = (float)(1.0 - g * g);
    S.hg_b[k] = (float)(1.0 - g);
    S.hg_c[k] = iso ? 0.0f : (float)(2.0 * g);
    S.hg_1pg2[k] = (float)(1.0 + g * g);
    S.hg_inv2g[k] = iso ? 0.0f : (float)(0.5 / g);
    for (int s = 0; s < 2; ++s) {
      S.src_cdf_d[s][k] = P.src_cdf_d[s * kMaxFreq + k];
      S.src_alias[s][k] = P.src_alias[s * kMaxFreq + k];
      S.sed_lo[s][k] = 0u;
      S.sed_hi[s][k] = 0u;
    }
  }
  if (threadIdx.x < 2) {
    S.inj_lo[threadIdx.x] = S.inj_hi[threadIdx.x] = 0u;
    S.dir_lo[threadIdx.x] = S.dir_hi[threadIdx.x] = 0u;
  }
  if (threadIdx.x < CNT_COUNT) S.rare[threadIdx.x] = 0u;
  if (threadIdx.x < kMaxWarps) S.wq_next[threadIdx.x] = S.wq_end[threadIdx.x] = 0ull;
  for (int j = threadIdx.x; j < P.n_tnodes_pow2; j += blockDim.x) sLnode[j] = P.Lnode_f[j];
  for (int b = threadIdx.x; b < kGuide; b += blockDim.x) S.nguide[b] = P.nguide[b];
  if (threadIdx.x == 0) {
    S.g_b0 = P.nmeta[0];
    S.g_sh = P.nmeta[1];
    const unsigned long long seed = P.seed_dev ? *P.seed_dev : P.seed;
    S.key[0] = (uint32_t)seed;
    S.key[1] = (uint32_t)(seed >> 32);
  }
}

// End of a CTA's work: per-lane event counters and the CTA's shared-memory
// tallies into the device counters (no warp collectives).
template <int PREC>
__device__ __forceinline__ void flush_tallies(const TransportParams &P, Shared &S, const Tally &T) {
  if (T.cross) atomicAdd(&S.rare[CNT_CROSS], T.cross);
  if (T.scat) atomicAdd(&S.rare[CNT_SCATTER], T.scat);
  if (T.abs) atomicAdd(&S.rare[CNT_ABSORB], T.abs);
  if constexpr (PREC == PREC_FP64) {
    if (T.e_inj != 0.0) atomicAdd(P.energies + EN_INJECTED, T.e_inj);
    if (T.e_direct != 0.0) atomicAdd(P.energies + EN_DIRECT, T.e_direct);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < CNT_COUNT; i += blockDim.x)
    if (S.rare[i]) atomicAdd(P.counters + i, (unsigned long long)S.rare[i]);
  if (PREC != PREC_FP64 && P.n_models == 1) {
    auto pair = [](unsigned int lo, unsigned int hi) { return ((unsigned long long)hi << 32) | lo; };
    for (int i = threadIdx.x; i < 2 * kMaxFreq; i += blockDim.x) {
      const unsigned long long v = pair(S.sed_lo[i >> 6][i & 63], S.sed_hi[i >> 6][i & 63]);
      if (v) atomicAdd(P.sed_q + i, v);
    }
    if (threadIdx.x < 2) {
      const unsigned long long vi = pair(S.inj_lo[threadIdx.x], S.inj_hi[threadIdx.x]);
      const unsigned long long vd = pair(S.dir_lo[threadIdx.x], S.dir_hi[threadIdx.x]);
      if (vi) atomicAdd(P.inj_q + threadIdx.x, vi);
      if (vd) atomicAdd(P.dir_q + threadIdx.x, vd);
    }
  }
}

// Whether the move that stopped a lane crossed a boundary: the exit (from
// the cloud, or from the forced pre-walk's range) does, an interaction in
// the cell does not.
template <int OPT>
__device__ __forceinline__ bool stop_crossed(const Lane<float> &L) {
  if constexpr ((OPT & OPT_NOFFI) != 0) return L.st == ST_ESCAPE;
  else return L.st == L.exit_st;
}

// The FP32 move of the staged-geometry kernels (OPT_SGEO): the same
// arithmetic as boundary() + move(), with the current cell's record and
// density (G, rho) carried in registers and the next cell's fetched from
// shared memory as soon as the next cell is known, so that the load overlaps
// the rest of the crossing instead of opening the next one (measured +1 to
// +3 % with the block counting below).  CC: the caller counts the block's
// crossings.
template <int OPT, bool CC>
__device__ __forceinline__ void move_staged(const TransportParams &P, Lane<float> &L, Tally &T, const float4 *sg,
                                            const float *sr, float4 &G, float &rho) {
  const int c = L.cell;
  const float d_in = (G.x - L.p2) + G.y;
  const bool inward = (L.s < 0.0f) & (d_in > 0.0f);
  const float d = fmaxf(inward ? d_in : (G.z - L.p2) + G.w, 1.0e-36f);
  const int next = inward ? c - 1 : c + 1;
  const float rho_c = rho;
  // next is in [-1, n] (the void, a shell, or out): the record fetched is in [0, n]
  int pi = L.gbase + min(next, L.n - 1);
  DIES_BOUND(P, pi >= 0 && pi < P.sgeo_n, STATUS_BAD_CELL, pi = 0);
  G = sg[pi];
  rho = sr[pi];
  const float sb = (inward ? -d : d) * rsqrt_ftz(d);
  const float l = sb - L.s;
  const float a2 = fmaf(rho_c, l, L.acc);
  if (a2 > L.lim) {
    L.s += fminf(__fdividef(L.lim - L.acc, rho_c), l);
    L.st = L.next_ev;
  } else {
    L.acc = a2;
    L.s = sb;
    L.cell = next;
    if constexpr ((OPT & OPT_NOFFI) != 0) {
      if constexpr (!CC) T.cross++;
      if (next >= L.n) L.st = ST_ESCAPE;
    } else {
      if constexpr (!CC) T.cross += L.cinc;
      if ((unsigned)(next - L.lo) >= (unsigned)L.span) L.st = L.exit_st;
    }
  }
}

// The FP32 forms are held to 48 registers (5 CTAs of 256 per SM): the
// forced-interaction state would otherwise cost a CTA per SM, which is worth
// more than the few spills in the rare-event path (measured).
template <int PREC, int MODE, bool RECORD, int OPT>
__global__ void __launch_bounds__(256, PREC == PREC_FP64 ? 1 : 5) k_transport(const TransportParams P) {
  using Real = typename RealOf<PREC>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Shared &S = *reinterpret_cast<Shared *>(smem_raw);
  constexpr bool kSG = (OPT & OPT_SGEO) != 0;
  float *sLnode = reinterpret_cast<float *>(smem_raw + sizeof(Shared) + (kSG ? sgeo_bytes(P.sgeo_n) : 0));

  stage_tables(P, S, sLnode);
  if constexpr (kSG) {
    float4 *sg = reinterpret_cast<float4 *>(smem_raw + sizeof(Shared));
    float *sr = reinterpret_cast<float *>(sg + P.sgeo_n);
    for (int j = threadIdx.x; j < P.sgeo_n; j += blockDim.x) {
      sg[j] = P.geo[j];
      sr[j] = P.rhoe[j];
    }
  }
  __syncthreads();

  Tally T;
  T.cross = T.scat = T.abs = 0;
  T.e_inj = T.e_direct = 0.0;

  bool timed_out = false;
  Lane<Real> L;
  L.st = ST_DEAD;
  const unsigned long long t0 = globaltimer();
  unsigned idle = 0;  // iterations since this warp last ran its rare path
  unsigned sections = 0;
  // All warp-wide decisions come from ballots taken by all 32 lanes; nothing
  // about the warp is carried between iterations.
  for (;;) {
    // up to P.inner moves per lane (in blocks of kCheck, P.inner rounded up);
    // a lane that parks skips the rest of its block (one divergent region per
    // block, not per move), and after each block the warp stops early once
    // batch_min lanes no longer move (warp-uniform loop)
    for (int k = 0; k < P.inner; k += kCheck) {
      if (L.st <= ST_FORCED) {
        // every move of a block crosses a boundary but the one that stops
        // the lane (an interaction in its cell; the exit from the cloud or
        // from the forced pre-walk's range does cross): the block's
        // crossings are counted once, from where it stopped, instead of at
        // each move (measured +1 to +2 %).  The forced-interaction forms
        // count them only in flights that count crossings (cw = L.cinc;
        // not the pre-walk), which cannot change within a block.
        constexpr bool kCC = PREC != PREC_FP64;
        const unsigned cw = ((OPT & OPT_NOFFI) != 0) ? 1u : (unsigned)L.cinc;
        if constexpr (kCC) T.cross += kCheck * cw;
        if constexpr (kSG && PREC != PREC_FP64) {
          const float4 *sg = reinterpret_cast<const float4 *>(smem_raw + sizeof(Shared));
          const float *sr = reinterpret_cast<const float *>(sg + P.sgeo_n);
          int ci = L.gbase + L.cell;
          DIES_BOUND(P, ci >= 0 && ci < P.sgeo_n, STATUS_BAD_CELL, ci = 0);
          float4 G = sg[ci];
          float rho = sr[ci];
#pragma unroll
          for (int j = 0; j < kCheck; ++j) {
            move_staged<OPT, kCC>(P, L, T, sg, sr, G, rho);
            if (L.st > ST_FORCED) {
              if constexpr (kCC) T.cross -= (kCheck - j - (stop_crossed<OPT>(L) ? 1 : 0)) * cw;
              break;
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < kCheck; ++j) {
            move<PREC, MODE, RECORD, OPT, kCC>(P, S, L, T);
            if (L.st > ST_FORCED) {
              if constexpr (kCC) T.cross -= (kCheck - j - (stop_crossed<OPT>(L) ? 1 : 0)) * cw;
              break;
            }
          }
        }
      }
      if (__popc(__ballot_sync(kFull, L.st > ST_FORCED)) >= P.batch_min) break;
    }
    const unsigned waiting = __ballot_sync(kFull, (unsigned)(L.st - ST_ESCAPE) <= (unsigned)(ST_DEAD - ST_ESCAPE));
    const unsigned done = __ballot_sync(kFull, L.st == ST_DONE);
    if (done == kFull) break;
    if ((waiting | done) != kFull && __popc(waiting) < P.batch_min) {
      if (++idle < kFlightLimit) continue;
      // watchdog: record the first stuck lane, end the moving packages as lost
      if (L.st <= ST_FORCED) {
        if (atomicCAS(P.diag, 0u, 1u) == 0u) {
          P.diag[1] = (uint32_t)L.st;
          P.diag[2] = (uint32_t)L.cell;
          P.diag[3] = (uint32_t)L.f;
          P.diag[4] = (uint32_t)L.n;
          P.diag[5] = __float_as_uint((float)L.s);
          P.diag[6] = __float_as_uint((float)L.p2);
          if constexpr (PREC == PREC_FP64) {
            P.diag[7] = __float_as_uint((float)L.tauA);
            P.diag[8] = __float_as_uint((float)L.tauS);
          } else {
            P.diag[7] = __float_as_uint(L.acc);
            P.diag[8] = __float_as_uint(L.lim);
          }
          P.diag[9] = __float_as_uint((float)L.ka);
          P.diag[10] = __float_as_uint((float)L.ks);
          P.diag[11] = __float_as_uint((float)L.w);
          P.diag[12] = L.pkg_lo;
          P.diag[13] = (uint32_t)L.model;
          __threadfence();
        }
        lose<RECORD>(P, S, L, CNT_KILL_CAP);
        atomicOr(P.status, STATUS_STUCK);
      }
    }
    idle = 0;
    if (L.st == ST_ESCAPE) escape<PREC, RECORD>(P, S, L);
    // refill the finished lanes from the warp's chunk of work items
    refill<PREC, RECORD>(P, S, L);
    if ((unsigned)(L.st - ST_SCATTER) <= (unsigned)(ST_FFIEND - ST_SCATTER)) rare<PREC, MODE, RECORD, OPT>(P, S, sLnode, L, T);
    if ((++sections & 31u) == 0 && L.st != ST_DONE && (globaltimer() - t0) > P.time_budget_ns) {
      // time budget reached: this lane gives up its package and its share of the work
      atomicOr(P.status, STATUS_TIMEOUT);
      L.st = ST_DONE;
      timed_out = true;
    }
  }
  if (!timed_out && L.st != ST_DONE) atomicOr(P.status, STATUS_ABANDONED);

  flush_tallies<PREC>(P, S, T);
}

// ------------------------------------------ two packages per thread (pool)
// An option of the FP32 forms without forced first interaction (launch knob
// packages_per_thread = 2).  Besides the package in its registers, every
// lane owns two slots of a per-warp pool of 64 packages in shared memory.
// A lane whose package stops for a scattering, an absorption or a start
// leaves it in an empty slot and takes a package that is ready to move, so
// the lanes of the warp keep crossing boundaries; the waiting events are
// then run in passes of ONE kind, with as many lanes as the pool holds
// events of that kind (the kind the warp can serve most of), instead of the
// few lanes of each kind that happen to stop together.  Slot bookkeeping is
// warp-synchronous: lane l keeps the kind of slots l and l + 32 in registers
// (the State of the stored package, or kEmpty), and every assignment of
// lanes to slots is derived from ballots by all 32 lanes.  No wait depends
// on another warp.
constexpr int kPool = 64;   // package slots per warp
constexpr int kEmpty = 15;  // kind of an empty slot (else: the State of its package)

__device__ __forceinline__ bool is_event(int st) {
  return (unsigned)(st - ST_SCATTER) <= (unsigned)(ST_INJECT - ST_SCATTER);
}

// The state a package carries between events (FP32 forms, no forced
// interaction) as four float4 in structure-of-arrays order: slot i of group
// g at pool[g * kPool + i], so a warp's accesses to distinct slots do not
// share banks more than the 128-bit access pattern requires.
__device__ __forceinline__ void pool_put(float4 *pool, int slot, const Lane<float> &L) {
#ifdef DIES_CHECK
  if ((unsigned)slot >= (unsigned)kPool) return;  // (the caller's ballot arithmetic keeps it in range)
#endif
  const uint32_t meta =
      ((uint32_t)L.f & 63u) | ((uint32_t)L.src << 8) | ((uint32_t)L.st << 12) | ((uint32_t)L.next_ev << 16);
  pool[slot] = make_float4(L.p2, L.s, L.w, L.acc);
  pool[kPool + slot] = make_float4(L.lim, L.eps, __int_as_float(L.cell), __uint_as_float(meta));
  pool[2 * kPool + slot] =
      make_float4(__int_as_float(L.model), __int_as_float(L.gbase), __int_as_float(L.n), __int_as_float(L.n64));
  pool[3 * kPool + slot] =
      make_float4(__uint_as_float(L.events), __uint_as_float(L.blk), __uint_as_float(L.pkg_lo), __uint_as_float(L.pkg_hi));
}

__device__ __forceinline__ void pool_get(const float4 *pool, int slot, const Shared &S, Lane<float> &L) {
#ifdef DIES_CHECK
  if ((unsigned)slot >= (unsigned)kPool) slot = 0;
#endif
  const float4 a = pool[slot], b = pool[kPool + slot], c = pool[2 * kPool + slot], d = pool[3 * kPool + slot];
  L.p2 = a.x;
  L.s = a.y;
  L.w = a.z;
  L.acc = a.w;
  L.lim = b.x;
  L.eps = b.y;
  L.cell = __float_as_int(b.z);
  const uint32_t meta = __float_as_uint(b.w);
  L.f = (int)(meta & 63u);
  L.src = (int)((meta >> 8) & 15u);
  L.st = (int)((meta >> 12) & 15u);
  L.next_ev = (int)(meta >> 16);
  L.model = __float_as_int(c.x);
  L.gbase = __float_as_int(c.y);
  L.n = __float_as_int(c.z);
  L.n64 = __float_as_int(c.w);
  L.cell_off = L.gbase - L.model - 1;
  L.events = __float_as_uint(d.x);
  L.blk = __float_as_uint(d.y);
  L.pkg_lo = __float_as_uint(d.z);
  L.pkg_hi = __float_as_uint(d.w);
  L.ka = S.kabs_f[L.f];
  L.ks = S.ksca_f[L.f];
}

// slot of the r-th (from 0) set bit of the 64-bit slot mask (lo: slots 0-31)
__device__ __forceinline__ int nth_slot(unsigned lo, unsigned hi, int r) {
  const int nl = __popc(lo);
  return r < nl ? (int)__fns(lo, 0, r + 1) : 32 + (int)__fns(hi, 0, r - nl + 1);
}

// Slot-kind bookkeeping of an assignment: the first n set slots of (lo, hi)
// go, in order, to the first n lanes of src; each such slot takes the value
// val of its lane.  Called by all 32 lanes; lane l updates slots l, l + 32.
__device__ __forceinline__ void set_kinds(unsigned lo, unsigned hi, unsigned src, int n, int val, int &k0,
                                          int &k1) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  const int r0 = __popc(lo & below), r1 = __popc(lo) + __popc(hi & below);
  const bool a0 = ((lo >> lane) & 1u) && r0 < n, a1 = ((hi >> lane) & 1u) && r1 < n;
  const int v0 = __shfl_sync(kFull, val, a0 ? (int)__fns(src, 0, r0 + 1) : lane);
  const int v1 = __shfl_sync(kFull, val, a1 ? (int)__fns(src, 0, r1 + 1) : lane);
  if (a0) k0 = v0;
  if (a1) k1 = v1;
}
__device__ __forceinline__ void clear_kinds(unsigned lo, unsigned hi, int n, int &k0, int &k1) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  if (((lo >> lane) & 1u) && __popc(lo & below) < n) k0 = kEmpty;
  if (((hi >> lane) & 1u) && __popc(lo) + __popc(hi & below) < n) k1 = kEmpty;
}

// After a block of moves: escapes tallied, stopped packages left in empty
// slots, idle lanes given ready packages, finished lanes new work.
template <int PREC, int OPT>
__device__ __forceinline__ void pool_exchange(const TransportParams &P, Shared &S, float4 *pool, Lane<float> &L,
                                              int &k0, int &k1) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  if (L.st == ST_ESCAPE) escape<PREC, false>(P, S, L);
  const unsigned evl = __ballot_sync(kFull, is_event(L.st));
  if (evl != 0u) {
    const unsigned elo = __ballot_sync(kFull, k0 == kEmpty), ehi = __ballot_sync(kFull, k1 == kEmpty);
    const int n = min(__popc(evl), __popc(elo) + __popc(ehi));
    if (n > 0) {
      set_kinds(elo, ehi, evl, n, L.st, k0, k1);
      if ((evl >> lane) & 1u) {
        const int r = __popc(evl & below);
        if (r < n) {
          pool_put(pool, nth_slot(elo, ehi, r), L);
          L.st = ST_DEAD;
        }
      }
    }
  }
  const unsigned idl = __ballot_sync(kFull, L.st == ST_DEAD || L.st == ST_DONE);
  if (idl != 0u) {
    const unsigned rlo = __ballot_sync(kFull, k0 == ST_NORMAL), rhi = __ballot_sync(kFull, k1 == ST_NORMAL);
    const int n = min(__popc(idl), __popc(rlo) + __popc(rhi));
    if (n > 0) {
      if ((idl >> lane) & 1u) {
        const int r = __popc(idl & below);
        if (r < n) pool_get(pool, nth_slot(rlo, rhi, r), S, L);
      }
      clear_kinds(rlo, rhi, n, k0, k1);
    }
  }
  refill<PREC, false>(P, S, L);
  __syncwarp();
}

// One pass of a single event kind: the kind of which the warp can serve the
// most events now (those its lanes hold, plus those in slots that free or
// displaced lanes can take).  Other lanes' packages are moved into empty
// slots when the free lanes are too few.
template <int PREC, int OPT>
__device__ __forceinline__ void pool_pass(const TransportParams &P, Shared &S, const float *sLnode, float4 *pool,
                                          Lane<float> &L, Tally &T, int &k0, int &k1) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  if (L.st == ST_ESCAPE) escape<PREC, false>(P, S, L);  // (an exchange always comes first; kept for safety)
  const unsigned fre = __ballot_sync(kFull, L.st == ST_DEAD || L.st == ST_DONE);
  const unsigned elo = __ballot_sync(kFull, k0 == kEmpty), ehi = __ballot_sync(kFull, k1 == kEmpty);
  const int room = __popc(fre) + __popc(elo) + __popc(ehi);
  int kind = -1, best = 0;
  unsigned el = 0u, slo = 0u, shi = 0u;
#pragma unroll
  for (int e = ST_SCATTER; e <= ST_INJECT; ++e) {
    const unsigned l = __ballot_sync(kFull, L.st == e);
    const unsigned a = __ballot_sync(kFull, k0 == e), b = __ballot_sync(kFull, k1 == e);
    const int served = __popc(l) + min(__popc(a) + __popc(b), min(room, 32 - __popc(l)));
    if (served > best) {
      best = served;
      kind = e;
      el = l;
      slo = a;
      shi = b;
    }
  }
  if (kind < 0) return;
  const int want = min(__popc(slo) + __popc(shi), 32 - __popc(el));
  const unsigned oth = ~(el | fre);
  const int ndisp = min(max(want - __popc(fre), 0), min(__popc(oth), __popc(elo) + __popc(ehi)));
  if (ndisp > 0) {
    set_kinds(elo, ehi, oth, ndisp, L.st, k0, k1);
    if ((oth >> lane) & 1u) {
      const int r = __popc(oth & below);
      if (r < ndisp) {
        pool_put(pool, nth_slot(elo, ehi, r), L);
        L.st = ST_DEAD;
      }
    }
  }
  const unsigned fr2 = __ballot_sync(kFull, L.st == ST_DEAD || L.st == ST_DONE);
  const int nload = min(want, __popc(fr2));
  if (nload > 0) {
    if ((fr2 >> lane) & 1u) {
      const int r = __popc(fr2 & below);
      if (r < nload) pool_get(pool, nth_slot(slo, shi, r), S, L);
    }
    clear_kinds(slo, shi, nload, k0, k1);
  }
  __syncwarp();
  if (L.st == kind) rare<PREC, MODE_IRE, false, OPT>(P, S, sLnode, L, T);
  __syncwarp();
}

template <int PREC, int OPT>
__global__ void __launch_bounds__(256, 4) k_transport_pool(const TransportParams P) {
  static_assert(PREC != PREC_FP64 && (OPT & OPT_NOFFI) != 0, "pool variant: FP32 forms without forced interaction");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Shared &S = *reinterpret_cast<Shared *>(smem_raw);
  float *sLnode = reinterpret_cast<float *>(smem_raw + sizeof(Shared));
  float4 *pool = reinterpret_cast<float4 *>(smem_raw + pool_offset(P.n_tnodes_pow2)) + (threadIdx.x >> 5) * (4 * kPool);
  stage_tables(P, S, sLnode);
  __syncthreads();

  Tally T;
  T.cross = T.scat = T.abs = 0;
  T.e_inj = T.e_direct = 0.0;
  Lane<float> L;
  L.st = ST_DEAD;
  int k0 = kEmpty, k1 = kEmpty;
  const unsigned long long t0 = globaltimer();
  unsigned quiet = 0, sections = 0;
  bool timed_out = false;
  for (;;) {
    bool pass = false;
    for (int k = 0; k < P.inner; k += kCheck) {
      const bool was_moving = L.st <= ST_FORCED;
      if (was_moving) {
#pragma unroll
        for (int j = 0; j < kCheck; ++j) {
          move<PREC, MODE_IRE, false, OPT>(P, S, L, T);
          if (L.st > ST_FORCED) break;
        }
      }
      // the flight watchdog counts blocks in which moving lanes moved but none stopped
      if (__ballot_sync(kFull, was_moving && L.st > ST_FORCED) != 0u) quiet = 0;
      else if (__ballot_sync(kFull, was_moving) != 0u) ++quiet;
      if (__ballot_sync(kFull, L.st > ST_FORCED) == 0u) continue;
      pool_exchange<PREC, OPT>(P, S, pool, L, k0, k1);
      const int empty = __popc(__ballot_sync(kFull, k0 == kEmpty)) + __popc(__ballot_sync(kFull, k1 == kEmpty));
      const int moving = __popc(__ballot_sync(kFull, L.st <= ST_FORCED));
      if (empty < P.batch_min || moving <= 32 - P.batch_min) {
        pass = true;
        break;
      }
    }
    if (__ballot_sync(kFull, L.st != ST_DONE) == 0u && __ballot_sync(kFull, k0 != kEmpty || k1 != kEmpty) == 0u)
      break;
    if (pass || __ballot_sync(kFull, L.st <= ST_FORCED) == 0u) pool_pass<PREC, OPT>(P, S, sLnode, pool, L, T, k0, k1);
    if (quiet >= kFlightLimit) {
      // watchdog: kFlightLimit blocks of moves without a stop; end the moving packages as lost
      if (L.st <= ST_FORCED) {
        lose<false>(P, S, L, CNT_KILL_CAP);
        atomicOr(P.status, STATUS_STUCK);
      }
      quiet = 0;
    }
    if ((++sections & 31u) == 0 && (globaltimer() - t0) > P.time_budget_ns) {
      // time budget reached: this warp gives up its packages and its share of the work
      atomicOr(P.status, STATUS_TIMEOUT);
      L.st = ST_DONE;
      k0 = k1 = kEmpty;
      timed_out = true;
    }
  }
  if (!timed_out && L.st != ST_DONE) atomicOr(P.status, STATUS_ABANDONED);
  flush_tallies<PREC>(P, S, T);
}

// FP32 forms: convert the fixed-point tallies of every model to energies
// (one block of 64 threads per model).
__global__ void k_tally(const ModelDesc *desc, unsigned long long n_per_source, const unsigned long long *sed_q,
                        const unsigned long long *inj_q, const unsigned long long *dir_q, double *sed,
                        double *energies, int rep) {
  const int m = blockIdx.x, k = threadIdx.x, nm = gridDim.x;
  const double unit = 1.0 / (double)kQuantum;
  const double e0 = desc[m].L[0] / (double)n_per_source, e1 = desc[m].L[1] / (double)n_per_source;
  unsigned long long s0 = 0, s1 = 0, i0 = 0, i1 = 0, d0 = 0, d1 = 0;  // integer sums over the replicas
  for (int r = 0; r < rep; ++r) {
    const size_t mr = (size_t)r * nm + m;
    s0 += sed_q[mr * 2 * kMaxFreq + k];
    s1 += sed_q[mr * 2 * kMaxFreq + kMaxFreq + k];
    if (k == 0) {
      i0 += inj_q[2 * mr];
      i1 += inj_q[2 * mr + 1];
      d0 += dir_q[2 * mr];
      d1 += dir_q[2 * mr + 1];
    }
  }
  sed[(size_t)m * kMaxFreq + k] = ((double)s0 * e0 + (double)s1 * e1) * unit;
  if (k == 0) {
    const double inj = ((double)i0 * e0 + (double)i1 * e1) * unit;
    const double dir = ((double)d0 * e0 + (double)d1 * e1) * unit;
    if (inj != 0.0) atomicAdd(energies + EN_INJECTED, inj);
    if (dir != 0.0) atomicAdd(energies + EN_DIRECT, dir);
  }
}

// Temperature of every cell from its absorbed energy: log-log interpolation
// of T(Lambda) between table nodes; below the first node T_min, above the
// last T_max.
// E and Ecur hold cell c at c * kEStride and c * kCStride (the spread IRE
// accumulators); the FP64 forms' energies are also written to E_out packed.
__global__ void k_finalize(int n_cells, const double *E, const float *Eprev, const float *Ecur, int fp32,
                           const double *inv_mass, const double *Lnode, const double *lnT, int n, double *T_out,
                           double *E_out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  const double Ec = fp32 ? (double)(Eprev[c] + Ecur[(size_t)c * kCStride]) : E[(size_t)c * kEStride];
  if (!fp32) E_out[c] = Ec;
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
    float *cur = Ecur + (size_t)c * kCStride;  // spread counter (kCStride)
    Eprev[c] += *cur;
    *cur = 0.0f;
  }
}

// Work chunk of a warp: about 1/divisor of a warp's share of the launch
// (default 1/64), so that the last chunks (at most kChunkMax / 32 packages
// per lane) end close together while the device work counter sees few atomics.
constexpr unsigned long long kChunkMin = 32, kChunkMax = 1024;
unsigned chunk_size(unsigned long long total, int grid, int block, unsigned divisor) {
  const unsigned long long warps = (unsigned long long)grid * (unsigned long long)(block / 32);
  unsigned long long c = total / (warps * (unsigned long long)(divisor ? divisor : 64u) + 1ull);
  c = c < kChunkMin ? kChunkMin : (c > kChunkMax ? kChunkMax : c);
  return (unsigned)(c & ~31ull);
}

template <int PREC, int MODE, bool RECORD, int OPT = 0>
cudaError_t launch_one(const TransportParams &P, int grid, int block, size_t smem, cudaStream_t st) {
  auto kern = k_transport<PREC, MODE, RECORD, OPT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  TransportParams Q = P;
  Q.chunk = chunk_size(P.total, grid, block, P.refill_div);
  kern<<<grid, block, smem, st>>>(Q);
  launch_counter_add(1);
  return cudaGetLastError();
}

template <int PREC, int OPT>
cudaError_t launch_pool(const TransportParams &P, int grid, int block, size_t smem, cudaStream_t st) {
  auto kern = k_transport_pool<PREC, OPT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  TransportParams Q = P;
  Q.chunk = chunk_size(P.total, grid, block, P.refill_div);
  kern<<<grid, block, smem, st>>>(Q);
  launch_counter_add(1);
  return cudaGetLastError();
}

template <int PREC, int OPT>
cudaError_t occupancy_pool(int block, size_t smem, int *blocks_per_sm) {
  auto kern = k_transport_pool<PREC, OPT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, block, smem);
}

template <int PREC, int MODE, bool RECORD, int OPT = 0>
cudaError_t occupancy_one(int block, size_t smem, int *blocks_per_sm) {
  auto kern = k_transport<PREC, MODE, RECORD, OPT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, block, smem);
}

// IRE kernels of the FP32 forms: the OPT_PLAIN variant when every weighting
// option it drops is neutral, with sgeo_n > 0 (single model, no FP64
// crossings) the variant with the geometry staged in shared memory, and
// (launch_ire) the OPT_AGG variant when the launch aggregates its atomics
template <int PREC, int OPT>
cudaError_t launch_ire_a(const TransportParams &P, bool plain, int grid, int block, size_t smem, cudaStream_t st) {
  if constexpr ((OPT & (OPT_BATCH | OPT_R64)) == 0) {
    if (P.sgeo_n > 0) {
      const size_t sm = smem + sgeo_bytes(P.sgeo_n);
      return plain ? launch_one<PREC, MODE_IRE, false, OPT | OPT_PLAIN | OPT_SGEO>(P, grid, block, sm, st)
                   : launch_one<PREC, MODE_IRE, false, OPT | OPT_SGEO>(P, grid, block, sm, st);
    }
  }
  return plain ? launch_one<PREC, MODE_IRE, false, OPT | OPT_PLAIN>(P, grid, block, smem, st)
               : launch_one<PREC, MODE_IRE, false, OPT>(P, grid, block, smem, st);
}

template <int PREC, int OPT>
cudaError_t launch_ire(const TransportParams &P, bool plain, int grid, int block, size_t smem, cudaStream_t st) {
  return P.agg ? launch_ire_a<PREC, OPT | OPT_AGG>(P, plain, grid, block, smem, st)
               : launch_ire_a<PREC, OPT>(P, plain, grid, block, smem, st);
}

template <int PREC, int OPT>
cudaError_t occupancy_ire_a(bool plain, int sgeo_n, int block, size_t smem, int *blocks_per_sm) {
  if constexpr ((OPT & (OPT_BATCH | OPT_R64)) == 0) {
    if (sgeo_n > 0) {
      const size_t sm = smem + sgeo_bytes(sgeo_n);
      return plain ? occupancy_one<PREC, MODE_IRE, false, OPT | OPT_PLAIN | OPT_SGEO>(block, sm, blocks_per_sm)
                   : occupancy_one<PREC, MODE_IRE, false, OPT | OPT_SGEO>(block, sm, blocks_per_sm);
    }
  }
  return plain ? occupancy_one<PREC, MODE_IRE, false, OPT | OPT_PLAIN>(block, smem, blocks_per_sm)
               : occupancy_one<PREC, MODE_IRE, false, OPT>(block, smem, blocks_per_sm);
}

template <int PREC, int OPT>
cudaError_t occupancy_ire(bool plain, bool agg, int sgeo_n, int block, size_t smem, int *blocks_per_sm) {
  return agg ? occupancy_ire_a<PREC, OPT | OPT_AGG>(plain, sgeo_n, block, smem, blocks_per_sm)
             : occupancy_ire_a<PREC, OPT>(plain, sgeo_n, block, smem, blocks_per_sm);
}

}  // namespace

// the same decisions the kernels take on these fields (see OPT_PLAIN)
bool plain_weighting(const TransportParams &P) {
  return P.k_S_f == 1.0f && P.kA_f == nullptr && !P.scat_w && !P.remit_random && P.g_E_f == 0.0f;
}

size_t transport_smem_bytes(int n_tnodes_pow2) { return sizeof(Shared) + sizeof(float) * (size_t)n_tnodes_pow2; }

// the pool variant: the per-warp package pools after the tables (16-byte aligned)
size_t transport_smem_bytes_pool(int n_tnodes_pow2, int block) {
  return pool_offset(n_tnodes_pow2) + (size_t)(block / 32) * 4 * kPool * sizeof(float4);
}

// prec: PREC_*, mode: MODE_*.  The re-emitting frozen mode exists in the
// FP64 form only; the absorb-terminal mode also in the FP32 forms (single
// model, no per-package records), for the pure-absorber closed forms.
cudaError_t launch_transport(int prec, int mode, bool record, const TransportParams &P, int grid, int block,
                             cudaStream_t st) {
  const size_t smem = transport_smem_bytes(P.n_tnodes_pow2);
  if (mode == MODE_FROZEN_TERMINAL && prec != PREC_FP64) {
    if (record || P.n_models != 1) return cudaErrorInvalidValue;
    constexpr int TM = MODE_FROZEN_TERMINAL;
    if (prec == PREC_MIXED) {
      if (P.ffi)
        return P.r64 ? launch_one<PREC_MIXED, TM, false, OPT_R64>(P, grid, block, smem, st)
                     : launch_one<PREC_MIXED, TM, false, 0>(P, grid, block, smem, st);
      return P.r64 ? launch_one<PREC_MIXED, TM, false, OPT_R64 | OPT_NOFFI>(P, grid, block, smem, st)
                   : launch_one<PREC_MIXED, TM, false, OPT_NOFFI>(P, grid, block, smem, st);
    }
    return P.ffi ? launch_one<PREC_FP32, TM, false, 0>(P, grid, block, smem, st)
                 : launch_one<PREC_FP32, TM, false, OPT_NOFFI>(P, grid, block, smem, st);
  }
  if (mode != MODE_IRE) {
    if (prec != PREC_FP64) return cudaErrorInvalidValue;
    if (mode == MODE_FROZEN)
      return record ? launch_one<PREC_FP64, MODE_FROZEN, true>(P, grid, block, smem, st)
                    : launch_one<PREC_FP64, MODE_FROZEN, false>(P, grid, block, smem, st);
    return record ? launch_one<PREC_FP64, MODE_FROZEN_TERMINAL, true>(P, grid, block, smem, st)
                  : launch_one<PREC_FP64, MODE_FROZEN_TERMINAL, false>(P, grid, block, smem, st);
  }
  const bool batch = P.n_models > 1 && !P.r64;  // batches run their own variants (grouped tallies)
  const bool plain = plain_weighting(P);
  if (P.pool && !P.ffi && prec != PREC_FP64) {
    // two packages per thread: the pool variants (no forced interaction)
    const size_t sp = transport_smem_bytes_pool(P.n_tnodes_pow2, block);
    constexpr int NF = OPT_NOFFI;
    if (prec == PREC_MIXED) {
      if (batch) return launch_pool<PREC_MIXED, NF | OPT_BATCH>(P, grid, block, sp, st);
      return P.r64 ? launch_pool<PREC_MIXED, NF | OPT_R64>(P, grid, block, sp, st)
                   : launch_pool<PREC_MIXED, NF>(P, grid, block, sp, st);
    }
    return batch ? launch_pool<PREC_FP32, NF | OPT_BATCH>(P, grid, block, sp, st)
                 : launch_pool<PREC_FP32, NF>(P, grid, block, sp, st);
  }
  switch (prec) {
    case PREC_MIXED:
      if (batch)
        return P.ffi ? launch_ire<PREC_MIXED, OPT_BATCH>(P, plain, grid, block, smem, st)
                     : launch_ire<PREC_MIXED, OPT_BATCH | OPT_NOFFI>(P, plain, grid, block, smem, st);
      if (P.ffi)
        return P.r64 ? launch_ire<PREC_MIXED, OPT_R64>(P, plain, grid, block, smem, st)
                     : launch_ire<PREC_MIXED, 0>(P, plain, grid, block, smem, st);
      if (P.remit_cdf)
        return P.r64 ? launch_ire<PREC_MIXED, OPT_R64 | OPT_NOFFI | OPT_CDF>(P, plain, grid, block, smem, st)
                     : launch_ire<PREC_MIXED, OPT_NOFFI | OPT_CDF>(P, plain, grid, block, smem, st);
      return P.r64 ? launch_ire<PREC_MIXED, OPT_R64 | OPT_NOFFI>(P, plain, grid, block, smem, st)
                   : launch_ire<PREC_MIXED, OPT_NOFFI>(P, plain, grid, block, smem, st);
    case PREC_FP32:
      if (batch)
        return P.ffi ? launch_ire<PREC_FP32, OPT_BATCH>(P, plain, grid, block, smem, st)
                     : launch_ire<PREC_FP32, OPT_BATCH | OPT_NOFFI>(P, plain, grid, block, smem, st);
      return P.ffi ? launch_ire<PREC_FP32, 0>(P, plain, grid, block, smem, st)
                   : launch_ire<PREC_FP32, OPT_NOFFI>(P, plain, grid, block, smem, st);
    default: return launch_one<PREC_FP64, MODE_IRE, false>(P, grid, block, smem, st);
  }
}

cudaError_t transport_occupancy(int prec, int mode, int block, int n_tnodes_pow2, bool r64, bool ffi, bool batch,
                                bool pool, bool plain, bool agg, int sgeo_n, int *blocks_per_sm) {
  const size_t smem = transport_smem_bytes(n_tnodes_pow2);
  if (pool && mode == MODE_IRE && !ffi && prec != PREC_FP64) {
    const size_t sp = transport_smem_bytes_pool(n_tnodes_pow2, block);
    constexpr int NF = OPT_NOFFI;
    const bool b = batch && !r64;
    if (prec == PREC_MIXED) {
      if (b) return occupancy_pool<PREC_MIXED, NF | OPT_BATCH>(block, sp, blocks_per_sm);
      return r64 ? occupancy_pool<PREC_MIXED, NF | OPT_R64>(block, sp, blocks_per_sm)
                 : occupancy_pool<PREC_MIXED, NF>(block, sp, blocks_per_sm);
    }
    return b ? occupancy_pool<PREC_FP32, NF | OPT_BATCH>(block, sp, blocks_per_sm)
             : occupancy_pool<PREC_FP32, NF>(block, sp, blocks_per_sm);
  }
  if (mode == MODE_FROZEN_TERMINAL && prec != PREC_FP64) {
    constexpr int TM = MODE_FROZEN_TERMINAL;
    if (prec == PREC_MIXED) {
      if (ffi)
        return r64 ? occupancy_one<PREC_MIXED, TM, false, OPT_R64>(block, smem, blocks_per_sm)
                   : occupancy_one<PREC_MIXED, TM, false, 0>(block, smem, blocks_per_sm);
      return r64 ? occupancy_one<PREC_MIXED, TM, false, OPT_R64 | OPT_NOFFI>(block, smem, blocks_per_sm)
                 : occupancy_one<PREC_MIXED, TM, false, OPT_NOFFI>(block, smem, blocks_per_sm);
    }
    return ffi ? occupancy_one<PREC_FP32, TM, false, 0>(block, smem, blocks_per_sm)
               : occupancy_one<PREC_FP32, TM, false, OPT_NOFFI>(block, smem, blocks_per_sm);
  }
  if (mode != MODE_IRE) return occupancy_one<PREC_FP64, MODE_FROZEN, true>(block, smem, blocks_per_sm);
  if (batch && !r64 && prec == PREC_MIXED)
    return ffi ? occupancy_ire<PREC_MIXED, OPT_BATCH>(plain, agg, sgeo_n, block, smem, blocks_per_sm)
               : occupancy_ire<PREC_MIXED, OPT_BATCH | OPT_NOFFI>(plain, agg, sgeo_n, block, smem, blocks_per_sm);
  if (batch && prec == PREC_FP32)
    return ffi ? occupancy_ire<PREC_FP32, OPT_BATCH>(plain, agg, sgeo_n, block, smem, blocks_per_sm)
               : occupancy_ire<PREC_FP32, OPT_BATCH | OPT_NOFFI>(plain, agg, sgeo_n, block, smem, blocks_per_sm);
  switch (prec) {
    case PREC_MIXED:
      if (ffi)
        return r64 ? occupancy_ire<PREC_MIXED, OPT_R64>(plain, agg, sgeo_n, block, smem, blocks_per_sm)
                   : occupancy_ire<PREC_MIXED, 0>(plain, agg, sgeo_n, block, smem, blocks_per_sm);
      return r64 ? occupancy_ire<PREC_MIXED, OPT_R64 | OPT_NOFFI>(plain, agg, sgeo_n, block, smem, blocks_per_sm)
                 : occupancy_ire<PREC_MIXED, OPT_NOFFI>(plain, agg, sgeo_n, block, smem, blocks_per_sm);
    case PREC_FP32:
      return ffi ? occupancy_ire<PREC_FP32, 0>(plain, agg, sgeo_n, block, smem, blocks_per_sm)
                 : occupancy_ire<PREC_FP32, OPT_NOFFI>(plain, agg, sgeo_n, block, smem, blocks_per_sm);
    default: return occupancy_one<PREC_FP64, MODE_IRE, false>(block, smem, blocks_per_sm);
  }
}

cudaError_t launch_tally(cudaStream_t st, int n_models, const ModelDesc *desc, unsigned long long n_per_source,
                         const unsigned long long *sed_q, const unsigned long long *inj_q,
                         const unsigned long long *dir_q, double *sed, double *energies, int rep) {
  k_tally<<<n_models, kMaxFreq, 0, st>>>(desc, n_per_source, sed_q, inj_q, dir_q, sed, energies, rep);
  launch_counter_add(1);
  return cudaGetLastError();
}

cudaError_t launch_finalize(cudaStream_t st, int n_cells, const double *E, const float *Eprev, const float *Ecur,
                            int fp32, const double *inv_mass, const double *Lnode, const double *lnT, int n,
                            double *T_out, double *E_out) {
  const int tb = 256;
  k_finalize<<<(n_cells + tb - 1) / tb, tb, 0, st>>>(n_cells, E, Eprev, Ecur, fp32, inv_mass, Lnode, lnT, n, T_out,
                                                     E_out);
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
