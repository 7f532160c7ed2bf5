// dies_tables.cu -- device construction of the lookup tables of the IRE
// method: frequency bin widths, source-spectrum CDFs and luminosities, the
// emission table Lambda(T_j) and the difference-spectrum re-emission CDFs
// (Sect. 2.1 takes both the updated temperature and the re-emission frequency
// from precomputed tables), per-shell geometry and emission normalisation,
// and the per-shell spectra of the frozen pass.
// All table arithmetic is FP64; float copies are written for the FP32 paths.
#include "dies_common.cuh"

namespace dies {

namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kH = 6.62607015e-27;   // erg s
constexpr double kKB = 1.380649e-16;    // erg / K
constexpr double kC = 2.99792458e10;    // cm / s

__device__ __forceinline__ double planck(double nu, double T) {
  if (!(T > 0.0)) return 0.0;
  const double x = kH * nu / (kKB * T);
  if (x > 700.0) return 0.0;
  return 2.0 * kH * nu * nu * nu / (kC * kC) / expm1(x);
}

// Alias table over kMaxFreq slots (Walker's method, built with Vose's
// linear-time pairing of under- and over-full slots) for the distribution
// proportional to w[0..kMaxFreq) (uniform over the first F bins if all w are
// 0).  Entry: 26-bit acceptance threshold << 6 | alias bin.  One thread.
__device__ void build_alias(const double *w, int F, uint32_t *out) {
  double q[kMaxFreq], sum = 0.0;
  int small[kMaxFreq], large[kMaxFreq], ns = 0, nl = 0;
  uint32_t alias[kMaxFreq];
  for (int k = 0; k < kMaxFreq; ++k) sum += w[k];
  for (int k = 0; k < kMaxFreq; ++k) {
    const double p = (sum > 0.0) ? w[k] / sum : (k < F ? 1.0 / F : 0.0);
    q[k] = p * kMaxFreq;
    alias[k] = (uint32_t)k;
    if (q[k] < 1.0) small[ns++] = k; else large[nl++] = k;
  }
  // pair an under-full slot with an over-full bin that tops it up
  while (ns > 0 && nl > 0) {
    const int s = small[--ns], l = large[--nl];
    alias[s] = (uint32_t)l;
    q[l] = (q[l] + q[s]) - 1.0;
    if (q[l] < 1.0) small[ns++] = l; else large[nl++] = l;
  }
  // what is left is full up to rounding
  while (nl > 0) q[large[--nl]] = 1.0;
  while (ns > 0) q[small[--ns]] = 1.0;
  for (int k = 0; k < kMaxFreq; ++k) {
    uint32_t t;
    if (q[k] >= 1.0) {
      t = (1u << 26) - 1u;
      alias[k] = (uint32_t)k;
    } else {
      const double x = q[k] * 67108864.0;  // 2^26
      t = (x >= 67108863.0) ? (1u << 26) - 1u : (uint32_t)(x + 0.5);
    }
    out[k] = (t << 6) | alias[k];
  }
}

// inclusive scan over the 64 threads of a block (two warps); `sh` holds 2 doubles
__device__ double block64_inclusive_scan(double v, double *sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) sh[warp] = v;
  __syncthreads();
  if (warp == 1) v += sh[0];
  __syncthreads();
  return v;
}

// dnu_k = nu_k * (ln-nu width of bin k): half the ln distance to the two
// neighbours, the full distance to the only neighbour at the ends.
__device__ double bin_width(const double *nu, int F, int k) {
  double w;
  if (k == 0) w = log(nu[1]) - log(nu[0]);
  else if (k == F - 1) w = log(nu[F - 1]) - log(nu[F - 2]);
  else w = 0.5 * (log(nu[k + 1]) - log(nu[k - 1]));
  return nu[k] * w;
}

// One block of 64 threads: bin widths, source CDFs and the source spectral sums.
__global__ void k_freq_tables(int F, const double *nu, const double *J, const double *spec, double *dnu,
                              double *src_cdf_d, uint32_t *src_alias, double *src_sum) {
  __shared__ double sh[2];
  __shared__ double total;
  __shared__ double wsh[kMaxFreq];
  const int k = threadIdx.x;
  const double w = (k < F) ? bin_width(nu, F, k) : 0.0;
  dnu[k] = w;
  for (int s = 0; s < 2; ++s) {
    const double *src = (s == 0) ? J : spec;
    const double p = (src && k < F) ? src[k] * w : 0.0;
    const double c = block64_inclusive_scan(p, sh);
    if (k == 63) total = c;
    __syncthreads();
    const double T = total;
    __syncthreads();
    double v = (T > 0.0) ? c / T : (double)(k + 1) / F;
    if (k >= F - 1) v = 1.0;
    src_cdf_d[s * kMaxFreq + k] = v;
    if (k == 0) src_sum[s] = T;
    wsh[k] = p;
    __syncthreads();
    if (k == 0) build_alias(wsh, F, src_alias + s * kMaxFreq);
    __syncthreads();
  }
}

// One block per temperature node j (64 threads = frequencies):
//   Lambda_j = sum_k kabs_k B_k(T_j) dnu_k
//   row j of the re-emission CDF: difference spectrum kabs [B(T_j) - B(T_{j-1})] dnu
//   over the interval [Lambda_{j-1}, Lambda_j); row 0 covers [0, Lambda_0)
//   with the node-0 spectrum itself.
// Blocks j >= n pad the search tables with +inf up to a power of two.
__global__ void k_node_tables(int F, int n, double T_min, double T_max, const double *nu, const double *kabs,
                              const double *dnu, double *Lnode_d, float *Lnode_f, double *lnT, uint32_t *dalias,
                              double *dcdf_d, float *dcdf_f) {
  __shared__ double sh[2];
  __shared__ double total;
  __shared__ double wsh[kMaxFreq];
  const int j = blockIdx.x, k = threadIdx.x;
  if (j >= n) {
    if (k == 0) {
      Lnode_d[j] = __longlong_as_double(0x7ff0000000000000LL);
      Lnode_f[j] = __int_as_float(0x7f800000);
    }
    return;
  }
  const double step = log(T_max / T_min) / (double)(n - 1);
  const double Tj = T_min * exp(step * j);
  const double Tp = (j > 0) ? T_min * exp(step * (j - 1)) : 0.0;
  const double bj = (k < F) ? kabs[k] * planck(nu[k], Tj) * dnu[k] : 0.0;
  const double bp = (k < F && j > 0) ? kabs[k] * planck(nu[k], Tp) * dnu[k] : 0.0;
  // Lambda_j
  const double cj = block64_inclusive_scan(bj, sh);
  if (k == 63) total = cj;
  __syncthreads();
  if (k == 0) {
    Lnode_d[j] = total;
    Lnode_f[j] = (float)total;
    lnT[j] = log(Tj);
  }
  __syncthreads();
  // re-emission CDF row
  const double d = fmax(bj - bp, 0.0);
  const double c = block64_inclusive_scan(d, sh);
  if (k == 63) total = c;
  __syncthreads();
  const double tot = total;
  double v = (tot > 0.0) ? c / tot : (double)(k + 1) / F;
  if (k >= F - 1) v = 1.0;
  dcdf_d[(size_t)j * kMaxFreq + k] = v;
  dcdf_f[(size_t)j * kMaxFreq + k] = (float)v;  // FP32 forms with CDF rows (a launch option)
  wsh[k] = (k < F) ? d : 0.0;
  __syncthreads();
  if (k == 0) build_alias(wsh, F, dalias + (size_t)j * kMaxFreq);
}

// Guide table of the node search (FP32 forms): for a positive float e, the
// bucket b = (bits(e) - bits(Lambda_0)) >> shift (clamped to [0, kGuide)) is
// monotone in e; guide[b] = number of nodes with Lambda_j below the smallest
// e of bucket b, so the count of nodes <= e is reached from guide[b] by a
// short forward scan.  One block of kGuide threads.
__global__ void k_node_guide(int n, const float *Lnode_f, uint16_t *guide, int *meta) {
  const int b = threadIdx.x;
  const int b0 = __float_as_int(Lnode_f[0]);
  const int span = __float_as_int(Lnode_f[n - 1]) - b0;
  int sh = 0;
  while ((span >> sh) >= kGuide) ++sh;
  const float lo = __int_as_float(b0 + (b << sh));
  int c = 0;
  for (int j = 0; j < n; ++j) c += (Lnode_f[j] < lo) ? 1 : 0;
  guide[b] = (uint16_t)c;
  if (b == 0) {
    meta[0] = b0;
    meta[1] = sh;
  }
}

// Per-boundary R^2.
__global__ void k_boundaries(int n_bnd, const double *radii, double *r2d, float *r2f) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < n_bnd) {
    const double r = radii[b];
    r2d[b] = r * r;
    r2f[b] = (float)(r * r);
  }
}

// Per-cell density copies and emission normalisation 1/(4 pi rho V L_u^2),
// V the shell volume in length units; model luminosities.
__global__ void k_cells(int n_models, ModelDesc *desc, int n_cells_total, const double *radii, const double *rho,
                        double length_unit_cm, const double *src_sum, double L_point, double *rhod, float *rhof,
                        double *inv_mass, float *inv_massf) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n_models) {
    const double Rcm = desc[c].R * length_unit_cm;
    desc[c].L[0] = (desc[c].src_mask & 1) ? 4.0 * kPi * kPi * Rcm * Rcm * src_sum[0] : 0.0;
    desc[c].L[1] = (desc[c].src_mask & 2) ? L_point : 0.0;
    // 2^-64 L: the FP32 forms form the package energy L / N as this times
    // 2^64 / N (both factors exact powers of two apart), which keeps it
    // finite for luminosities above the float range
    desc[c].Lf[0] = (float)(desc[c].L[0] * 0x1p-64);
    desc[c].Lf[1] = (float)(desc[c].L[1] * 0x1p-64);
    desc[c].Rf = (float)desc[c].R;
  }
  if (c >= n_cells_total) return;
  // model of this cell (binary search over the cell offsets)
  int lo = 0, hi = n_models - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (desc[mid].cell_off <= c) lo = mid; else hi = mid - 1;
  }
  const int b = c + lo;  // boundaries of model lo start at cell_off + lo
  const double a = radii[b], r = radii[b + 1];
  const double V = 4.0 * kPi / 3.0 * (r - a) * (r * r + a * r + a * a);
  const double m = 4.0 * kPi * rho[c] * V * length_unit_cm * length_unit_cm;
  rhod[c] = rho[c];
  rhof[c] = (float)rho[c];
  inv_mass[c] = (m > 0.0) ? 1.0 / m : 0.0;
  inv_massf[c] = (m > 0.0) ? (float)(1.0 / m) : 0.0f;
}

// Per-cell geometry records of the FP32 transport, one per cell plus one for
// the central void in front of every model's cells (index bnd_off + cell + 1):
// {R_in^2 hi, R_in^2 lo, R_out^2 hi, R_out^2 lo} as float pairs (hi = float of
// the FP64 square, lo = float of the remainder) and the density (0 in the void).
__global__ void k_geo(int n_models, const ModelDesc *desc, int n_bnd, const double *radii, const double *rho,
                      float4 *geo, float *rhoe) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_bnd) return;
  int lo = 0, hi = n_models - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (desc[mid].bnd_off <= b) lo = mid; else hi = mid - 1;
  }
  const int i = b - desc[lo].bnd_off;  // 0 = void, i >= 1: cell i - 1
  const double ro2 = radii[b] * radii[b];
  const float rh = (float)ro2, rl = (float)(ro2 - (double)rh);
  float ih = 0.0f, il = 0.0f;
  if (i >= 1) {
    const double ri2 = radii[b - 1] * radii[b - 1];
    ih = (float)ri2;
    il = (float)(ri2 - (double)ih);
  }
  geo[b] = make_float4(ih, il, rh, rl);
  rhoe[b] = (i >= 1) ? (float)rho[b - lo - 1] : 0.0f;
}

// Frozen pass: per-cell CDF of kabs_k B_k(T_i) dnu_k (one block of 64 per cell).
__global__ void k_frozen_cdf(int F, const double *nu, const double *kabs, const double *dnu, const double *T,
                             double *cell_cdf) {
  __shared__ double sh[2];
  __shared__ double total;
  const int i = blockIdx.x, k = threadIdx.x;
  const double p = (k < F) ? kabs[k] * planck(nu[k], T[i]) * dnu[k] : 0.0;
  const double c = block64_inclusive_scan(p, sh);
  if (k == 63) total = c;
  __syncthreads();
  const double tot = total;
  double v = (tot > 0.0) ? c / tot : (double)(k + 1) / F;
  if (k >= F - 1) v = 1.0;
  cell_cdf[(size_t)i * kMaxFreq + k] = v;
}

}  // namespace

cudaError_t launch_freq_tables(cudaStream_t st, int F, const double *nu, const double *J, const double *spec,
                               double *dnu, double *src_cdf_d, uint32_t *src_alias, double *src_sum) {
  k_freq_tables<<<1, kMaxFreq, 0, st>>>(F, nu, J, spec, dnu, src_cdf_d, src_alias, src_sum);
  launch_counter_add(1);
  return cudaGetLastError();
}

cudaError_t launch_node_tables(cudaStream_t st, int F, int n, int n_pow2, double T_min, double T_max,
                               const double *nu, const double *kabs, const double *dnu, double *Lnode_d,
                               float *Lnode_f, double *lnT, uint32_t *dalias, double *dcdf_d, float *dcdf_f,
                               uint16_t *nguide, int *nmeta) {
  k_node_tables<<<n_pow2, kMaxFreq, 0, st>>>(F, n, T_min, T_max, nu, kabs, dnu, Lnode_d, Lnode_f, lnT, dalias,
                                             dcdf_d, dcdf_f);
  k_node_guide<<<1, kGuide, 0, st>>>(n, Lnode_f, nguide, nmeta);
  launch_counter_add(2);
  return cudaGetLastError();
}

cudaError_t launch_geometry(cudaStream_t st, int n_models, ModelDesc *desc, int n_cells_total, int n_bnd, const double *radii, const double *rho,
                            double length_unit_cm, const double *src_sum, double L_point, double *r2d, float *r2f,
                            double *rhod, float *rhof, double *inv_mass, float *inv_massf, float4 *geo, float *rhoe) {
  const int tb = 256;
  k_boundaries<<<(n_bnd + tb - 1) / tb, tb, 0, st>>>(n_bnd, radii, r2d, r2f);
  k_geo<<<(n_bnd + tb - 1) / tb, tb, 0, st>>>(n_models, desc, n_bnd, radii, rho, geo, rhoe);
  launch_counter_add(1);
  const int n = n_cells_total > n_models ? n_cells_total : n_models;
  k_cells<<<(n + tb - 1) / tb, tb, 0, st>>>(n_models, desc, n_cells_total, radii, rho, length_unit_cm, src_sum,
                                            L_point, rhod, rhof, inv_mass, inv_massf);
  launch_counter_add(2);
  return cudaGetLastError();
}

cudaError_t launch_frozen_cdf(cudaStream_t st, int n_cells, int F, const double *nu, const double *kabs,
                              const double *dnu, const double *T, double *cell_cdf) {
  k_frozen_cdf<<<n_cells, kMaxFreq, 0, st>>>(F, nu, kabs, dnu, T, cell_cdf);
  launch_counter_add(1);
  return cudaGetLastError();
}

}  // namespace dies
