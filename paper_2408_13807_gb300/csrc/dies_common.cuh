// dies_common.cuh -- device-side data layout and helpers shared by the
// kernels of the IRE library (tables, transport, temperature).
//
// Layout in HBM (one contiguous workspace per handle, 256-byte aligned
// segments; see workspace_layout() in dies_api.cu):
//   per model      ModelDesc (geometry offsets, source luminosities)
//   per boundary   R^2 as float and double (n_cells + 1 per model)
//   per cell       density (float, double), 1/(4 pi rho V L_u^2) (double),
//                  absorbed energy (double, or two floats for the FP32 form)
//   per frequency  dnu, kappa_abs, kappa_sca, g, source CDFs
//   per T node     Lambda_j = sum_k kappa_k B_k(T_j) dnu_k (float, double),
//                  ln T_j, and one re-emission CDF row of 64 entries
//                  (difference spectrum of the interval ending at node j)
// Everything the transport kernel reads per event is a few KB per model and
// stays in L1/L2; the per-frequency and per-node tables are staged in shared
// memory by every CTA.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dies {

constexpr int kMaxFreq = 64;
constexpr int kFreqShift = 6;  // row stride of the re-emission CDF table

enum Prec { PREC_MIXED = 0, PREC_FP32 = 1, PREC_FP64 = 2 };
enum Mode { MODE_IRE = 0, MODE_FROZEN = 1, MODE_FROZEN_TERMINAL = 2 };

// event codes folded into the per-package path hash
enum { EV_INJECT = 0, EV_CROSS = 1, EV_SCATTER = 2, EV_ABSORB = 3 };

// indices of the u64 counter block
enum {
  CNT_INJECTED = 0, CNT_ESCAPED, CNT_ABSORB, CNT_SCATTER, CNT_CROSS, CNT_KILL_WEIGHT, CNT_KILL_CAP,
  CNT_CLAMP_HI, CNT_FORCED, CNT_COUNT
};
// indices of the double energy block
enum { EN_INJECTED = 0, EN_LOST, EN_DIRECT, EN_COUNT };

// device status flags
enum : uint32_t {
  STATUS_TIMEOUT = 1u,
  STATUS_BAD_CELL = 2u,
  STATUS_BAD_FREQ = 4u,
  STATUS_STUCK = 8u,   // a warp ran kFlightLimit moves without a rare event; its moving lanes were ended
  STATUS_ABANDONED = 16u,  // a package was still in flight when its lane left the work loop
  STATUS_RANGE = 32u,      // all-FP32 form: an absorbed-energy counter left the FP32 range
  STATUS_BAD_ROW = 64u,    // check build: a table row, model or slot index out of range
};
constexpr uint32_t STATUS_BOUNDS = STATUS_BAD_CELL | STATUS_BAD_FREQ | STATUS_BAD_ROW;

// Device bounds checks of the check build (compiled with -DDIES_CHECK): an
// index outside its table sets a status flag (the run then reports
// DIES_ERANGE) and is clamped into range, so the access that follows stays
// in bounds.  No trap, no fault.  Compiled out otherwise.
#ifdef DIES_CHECK
#define DIES_BOUND(P, cond, flag, fix) \
  do {                                 \
    if (!(cond)) {                     \
      atomicOr((P).status, (flag));    \
      fix;                             \
    }                                  \
  } while (0)
#else
#define DIES_BOUND(P, cond, flag, fix) \
  do {                                 \
  } while (0)
#endif

// Consecutive loop iterations a warp may run without any lane finishing a
// flight segment; a legitimate flight crosses at most ~2 x shells boundaries.
constexpr unsigned kFlightLimit = 1u << 22;

struct alignas(16) ModelDesc {
  int cell_off;    // first cell of this model in the per-cell arrays
  int bnd_off;     // first boundary of this model in the per-boundary arrays
  int n_cells;
  int src_mask;    // bit 0: external field, bit 1: point source
  int n_src;
  int point_cell;  // start cell of point-source packages (-1 = central void)
  int n_fp64;      // MIXED form: cells [0, n_fp64) use FP64 crossing distances
  int pad0;
  double R;        // outer radius (length units)
  double L[2];     // source luminosities (erg/s), written by the table build
  unsigned long long pkg_off;  // first source slot of this model (slots x packages = work items)
  float Lf[2];     // 2^-64 x the luminosities, as float (FP32 forms: package energy = Lf x inv_n)
  float Rf;        // outer radius as float
  float pad1;
};

struct TransportParams {
  // geometry
  const ModelDesc *desc;
  int n_models;
  int F;
  const float *r2f;         // boundary radius^2
  const double *r2d;
  const float *rhof;        // cell density
  const double *rhod;
  const double *inv_mass;   // 1 / (4 pi rho V L_u^2)
  const float *inv_massf;
  const float4 *geo;        // FP32 forms: per cell + void {R_in^2 hi, lo, R_out^2 hi, lo}
  const float *rhoe;        // FP32 forms: density per geo record (0 in the void)
  // accumulators
  double *E;                // absorbed energy (MIXED / FP64 forms and frozen tallies)
  const float *Eprev;       // FP32 form: all previous batches (read only in a batch)
  float *Ecur;              // FP32 form: current batch
  double *sed;              // [n_models][kMaxFreq] (FP64 form writes it directly)
  // FP32 forms: fixed-point tallies, 2^-24 package energies per unit
  // fixed-point tallies of batches, in `rep` replicas (CTA b writes replica
  // b % rep) so that few models do not serialise on a few addresses
  unsigned long long *sed_q;  // [rep][n_models][2][kMaxFreq]
  unsigned long long *inj_q;  // [rep][n_models][2]
  unsigned long long *dir_q;  // [rep][n_models][2]
  int rep;                    // power of two
  // per-frequency tables
  const double *kabs_d, *ksca_d, *g_d;
  const double *src_cdf_d;  // [2][kMaxFreq]
  // temperature tables
  const double *Lnode_d;    // [n_tnodes]
  const float *Lnode_f;
  const uint32_t *dalias;   // FP32 forms: [n_tnodes][kMaxFreq] alias tables of the re-emission rows
  const uint32_t *src_alias;  // FP32 forms: [2][kMaxFreq] alias tables of the source spectra
  const uint16_t *nguide;   // FP32 forms: [kGuide] first node of each bucket of float(Lambda) bits
  const int *nmeta;         // {bits of Lambda_0, bucket shift}
  const double *dcdf_d;
  const float *dcdf_f;      // mixed form with remit_cdf: the re-emission CDF rows in FP32
  int n_tnodes;
  int n_tnodes_pow2;        // smallest power of two >= n_tnodes
  // frozen pass
  const double *cell_cdf;   // [n_cells][kMaxFreq]
  uint32_t *rec_events;     // [rows][3] or null
  unsigned long long *rec_hash;  // [rows] or null
  // work
  unsigned long long total;       // work items (packages) in this launch
  unsigned long long pkg_begin;   // first package index of every source in this launch
  unsigned long long pkg_len;     // packages per source in this launch
  unsigned long long n_per_source;  // packages per source in the whole run (sets eps)
  unsigned long long seed;
  const unsigned long long *seed_dev;  // if set, the seed is read from here (graph replays)
  unsigned long long *queue;
  unsigned long long *counters;   // [CNT_COUNT]
  double *energies;               // [EN_COUNT]
  uint32_t *status;
  uint32_t *diag;                 // [16]: diag[0] = 1 once filled; state of the first stuck lane
  // options
  double k_bg;
  int ffi;
  // weighted sampling beyond k_bg / FFI (Eqs. 6-8); kA_* null = no k_A weighting
  double g_E, g_S, k_S;
  int scat_w;
  const double *kA_d;       // per cell k_A (FP64 form)
  const float *kA_f;        // per cell k_A (FP32 forms)
  double kA_void;
  float g_E_f, g_S_f, k_S_f, kA_void_f;
  int remit_random;         // re-emit from a point uniform over the absorbing cell
  const double *radii_d;    // boundary radii (length units), boundary index cell_off + model + c
  int mode;
  unsigned long long max_events;
  unsigned long long time_budget_ns;
  float inv_n;      // 2^64 / n_per_source (FP32 package energies Lf x inv_n = L / N)
  double inv_nd;    // 1 / n_per_source in FP64
  float k_bg_f;     // k_bg as float (FP32 forms)
  int kbg_plain;    // k_bg == 1/2: no weighting
  int r64;          // MIXED form: some model has FP64 crossing distances in its inner shells
  int batch_min;    // lanes that must wait for a rare event before a warp runs them together
  int inner;        // moves per lane between two warp-collective sections (>= 1)
  unsigned chunk;   // work items a warp takes from the counter at a time (multiple of 32, >= 32; set at launch)
  unsigned refill_div;  // the chunk is about 1/refill_div of a warp's share of the launch (0 = 64)
  int agg;          // FP32 forms: warp-aggregated absorption atomics (lanes sharing a cell add once)
  int remit_cdf;    // mixed form, single model, no forced interaction: the kernel variant that
                    // searches FP32 CDF rows for the re-emission bin instead of alias rows
  int pool;         // FP32 forms without forced interaction: two packages per thread (per-warp pools)
  int e_stride;     // doubles between two cells' accumulators in E (IRE runs: kEStride, else 1)
  int c_stride;     // floats between two cells' counters in Ecur (IRE runs: kCStride, else 1)
  int sgeo_n;       // single-model IRE runs: geometry records staged in shared memory (0: read from L1/L2)
};

// Absorbed-energy accumulators of IRE runs, one per cell, each on its own
// 256-byte segment.  The absorptions of an optically thick model pile up in
// a few inner cells; packed 8 bytes apart, those cells' returning atomic adds
// all went to one L2 slice (measured: its atomic unit 65 % busy, the mean
// slice 0.5 %).  Spread, they are served by different slices: +68 % packages/s
// on the 1024-shell internal-source model, +28 % on C2 A_V = 100 (measured;
// 128-byte spacing gave most of it, 4 KB no more than 256 bytes).
constexpr int kAccSpreadBytes = 256;
constexpr int kEStride = kAccSpreadBytes / 8;  // FP64 accumulator E
constexpr int kCStride = kAccSpreadBytes / 4;  // FP32 current-batch counter Ecur

// Alias-table entries (FP32 forms): bits 6..31 the 26-bit acceptance
// threshold of the slot, bits 0..5 the alias bin; a slot that is full has
// itself as alias.
constexpr int kGuide = 1024;  // buckets of the node guide table

constexpr float kQuantum = 16777216.0f;  // 2^24 fixed-point units per package energy

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications by 0xD2511F53 / 0xCD9E8D57 with the high halves
// xored into the other words and the round key; the key advances by the Weyl
// increments 0x9E3779B9 / 0xBB67AE85 between rounds.
struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                       uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c0;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return U4{c0, c1, c2, c3};
}

// Per-package stream: key = seed, counter = (package lo, package hi, block, model ^ source << 24).
struct Stream {
  uint32_t k0, k1, c0, c1, c3;
  uint32_t blk;
  __device__ __forceinline__ U4 next() {
    U4 r = philox10(c0, c1, blk, c3, k0, k1);
    ++blk;
    return r;
  }
};

// double in (0,1): top 52 bits of a word pair, (m + 1/2) 2^-52 (exact, never 0 or 1)
__device__ __forceinline__ double u01d(uint32_t a, uint32_t b) {
  const unsigned long long m = ((unsigned long long)a << 20) | (unsigned long long)(b >> 12);
  return ((double)m + 0.5) * 0x1p-52;
}

// float in (0,1): 23 bits, (m + 1/2) 2^-23 (exact, never 0 or 1)
__device__ __forceinline__ float u01f(uint32_t m23) { return ((float)m23 + 0.5f) * 0x1p-23f; }
__device__ __forceinline__ float u01f_word(uint32_t w) { return u01f(w >> 9); }

// float in (0,1) with full relative precision near 0 (for 1 - mu^2 of the
// injection directions): (w + 1/2) 2^-32 rounded to float, capped below 1.
__device__ __forceinline__ float u01f_fine(uint32_t w) {
  float v = fmaf(__uint2float_rn(w), 0x1p-32f, 0x1p-33f);
  return fminf(v, 1.0f - 0x1p-24f);
}

// ---------------------------------------------------------------- FNV-1a
__device__ __forceinline__ unsigned long long fnv_word(unsigned long long h, uint32_t w) {
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    h ^= (unsigned long long)((w >> (8 * b)) & 0xffu);
    h *= 0x100000001b3ULL;
  }
  return h;
}
__device__ __forceinline__ uint32_t event_word(int ev, int cell, int f) {
  return (uint32_t)ev | ((uint32_t)(cell + 1) << 3) | ((uint32_t)f << 24);
}

// ----------------------------------------------------------- host helpers
void launch_counter_add(unsigned n);

}  // namespace dies
