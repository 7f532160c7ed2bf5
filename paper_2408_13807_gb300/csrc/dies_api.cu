// dies_api.cu -- host side of the C ABI declared in include/dies.h.
//
// A handle keeps host copies of its inputs, one device workspace holding every
// table and accumulator, and the results of its last run.  dies_run enqueues,
// on the handle's stream: (when inputs changed) the table-build kernels, the
// accumulator resets, the persistent transport kernel (N_B launches plus
// merges in the FP32 form) and the temperature kernel.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/dies.h"
#include "dies_common.cuh"

namespace dies {

// NVTX range over a host-side phase of a call (upload and table build,
// enqueue of the transport, wait and read-back), for timeline profilers;
// without a profiler attached the push and pop cost a few nanoseconds.
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range &) = delete;
  Range &operator=(const Range &) = delete;
};

static std::atomic<unsigned long long> g_launches{0};
void launch_counter_add(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

cudaError_t launch_freq_tables(cudaStream_t st, int F, const double *nu, const double *J, const double *spec,
                               double *dnu, double *src_cdf_d, uint32_t *src_alias, double *src_sum);
cudaError_t launch_node_tables(cudaStream_t st, int F, int n, int n_pow2, double T_min, double T_max,
                               const double *nu, const double *kabs, const double *dnu, double *Lnode_d,
                               float *Lnode_f, double *lnT, uint32_t *dalias, double *dcdf_d, float *dcdf_f,
                               uint16_t *nguide, int *nmeta);
cudaError_t launch_geometry(cudaStream_t st, int n_models, ModelDesc *desc, int n_cells_total, int n_bnd,
                            const double *radii, const double *rho, double length_unit_cm, const double *src_sum,
                            double L_point, double *r2d, float *r2f, double *rhod, float *rhof, double *inv_mass,
                            float *inv_massf, float4 *geo, float *rhoe);
cudaError_t launch_frozen_cdf(cudaStream_t st, int n_cells, int F, const double *nu, const double *kabs,
                              const double *dnu, const double *T, double *cell_cdf);
size_t transport_smem_bytes(int n_tnodes_pow2);
cudaError_t launch_transport(int prec, int mode, bool record, const TransportParams &P, int grid, int block,
                             cudaStream_t st);
cudaError_t transport_occupancy(int prec, int mode, int block, int n_tnodes_pow2, bool r64, bool ffi, bool batch,
                                bool pool, bool plain, bool agg, int sgeo_n, int *blocks_per_sm);
bool plain_weighting(const TransportParams &P);
cudaError_t launch_finalize(cudaStream_t st, int n_cells, const double *E, const float *Eprev, const float *Ecur,
                            int fp32, const double *inv_mass, const double *Lnode, const double *lnT, int n,
                            double *T_out, double *E_out);
cudaError_t launch_merge(cudaStream_t st, int n_cells, float *Eprev, float *Ecur);
cudaError_t launch_tally(cudaStream_t st, int n_models, const ModelDesc *desc, unsigned long long n_per_source,
                         const unsigned long long *sed_q, const unsigned long long *inj_q,
                         const unsigned long long *dir_q, double *sed, double *energies, int rep);

namespace {

thread_local std::string t_error;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_error = buf;
  return code;
}

#define DIES_CUDA(call)                                                                            \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(DIES_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int next_pow2(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

bool finite_nonneg(const double *a, int n) {
  for (int i = 0; i < n; ++i)
    if (!(std::isfinite(a[i]) && a[i] >= 0.0)) return false;
  return true;
}

// Offsets (bytes) of every segment of the device workspace.
struct Layout {
  size_t desc, radii, rho_in, r2d, r2f, rhod, rhof, inv_mass, inv_massf, kA_d, kA_f, geo, rhoe, E, Es, Eprev, Ecur, T, sed;
  size_t sed_q, inj_q, dir_q;
  size_t freq, kabs, ksca, g, J, spec, dnu, src_cdf_d, src_alias, src_sum;
  size_t Lnode_d, Lnode_f, lnT, dalias, dcdf_d, dcdf_f, nguide, nmeta;
  size_t counters, energies, queue, status, diag, seedw;
  size_t total;
};

}  // namespace

struct Problem {
  int n_models = 0;
  int n_cells = 0;  // total over models
  std::vector<ModelDesc> desc;
  std::vector<double> radii, rho;
  double length_unit_cm = 1.0;
  int F = 0;
  std::vector<double> freq, kabs, ksca, g;
  bool has_dust = false, has_sources = false;
  bool has_ext = false;
  std::vector<double> J, spec;
  double L_point = 0.0;
  std::vector<int> kind;  // per model: bit 0 external, bit 1 point (batch); 0 = follow the sources
  double k_bg = 0.5;
  int ffi = 0;
  double g_E = 0.0, g_S = 0.0, k_A = 1.0, k_S = 1.0, kA_lo = 3.0, kA_hi = 1.0;
  int scat_w = 0, kA_rho = 0, remit_random = 0;
  int prec = PREC_MIXED, n_batches = 1;
  double fp64_radius = 0.0;
  double T_min = 2.7, T_max = 1500.0;
  int n_tnodes = 1024;
  cudaStream_t stream = nullptr;
  int block = 256, blocks_per_sm = 0, rare_batch = 16, inner = 32, agg = 0;
  // package range of the next run (dies_set_package_range): packages
  // [range_first, range_first + range_count) of each source; resume keeps
  // the accumulators of the previous run
  bool range_set = false, range_resume = false;
  uint64_t range_first = 0, range_count = 0;
  int pkgs_per_thread = 1;  // 2: a second package per lane in per-warp shared-memory pools (FP32 forms, no FFI)
  int stage_geo = 1;  // launch knob: stage a single model's geometry in shared memory where it costs no CTA
  int sgeo_n = 0;  // geometry records the next IRE launch stages in shared memory (set by grid_for; 0: none)
  uint32_t last_grid = 0, last_block = 0, last_variant = 0;  // the launch grid_for chose (reported in dies_stats)
  int refill_div = 0;  // a warp takes ~1/refill_div of its share of the launch per trip to the work counter (0 = 64)
  int remit_table = DIES_TABLE_ALIAS;
  double time_budget_s = 120.0;
  // device
  unsigned char *ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_owned = false;
  Layout lay{};
  bool tables_valid = false;
  int sm_count = 0;
  // run timing: 0 start, 5 uploads done, 1 tables built, 2/3 around the transport, 4 end
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  bool events_ready = false;
  bool table_built_this_run = false;
  bool has_result = false;
  bool stats_pending = false;
  bool e_in_fp32_counters = false;  // the last run kept absorbed energies in the FP32 form's two counters
  unsigned long long launches_at_start = 0;
  dies_stats stats{};
  // a dies_run_frozen_static pass whose counters, status and SED still sit
  // in the library's static scratch (device addresses of those words)
  bool static_pending = false;
  const void *static_counters = nullptr, *static_energies = nullptr, *static_status = nullptr,
             *static_diag = nullptr, *static_sed = nullptr;
  // graph replay of the per-run device work (dies_set_graph)
  bool use_graph = false;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  unsigned long long *seed_host = nullptr;  // pinned; copied to the device by the graph
  struct GraphKey {
    TransportParams P;
    uint64_t n;
    int prec, n_batches, grid, block, n_cells, n_models, n_tnodes;
  };
  GraphKey gkey{};
  bool graph_valid = false;
  unsigned long long graph_kernels = 0;

  void drop_graph() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    gexec = nullptr;
    graph = nullptr;
    graph_valid = false;
  }

  ~Problem() {
    drop_graph();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (seed_host) cudaFreeHost(seed_host);
    if (ws_owned && ws) cudaFree(ws);
    for (auto &e : ev)
      if (e) cudaEventDestroy(e);
  }

  template <class T>
  T *at(size_t off) const { return reinterpret_cast<T *>(ws + off); }

  Layout layout() const {
    Layout L{};
    size_t o = 0;
    auto seg = [&](size_t bytes) {
      size_t r = o;
      o += align256(bytes);
      return r;
    };
    const size_t nb = (size_t)n_cells + n_models, nc = (size_t)n_cells, nm = (size_t)n_models;
    const size_t np2 = (size_t)next_pow2(n_tnodes), nt = (size_t)n_tnodes;
    L.desc = seg(nm * sizeof(ModelDesc));
    L.radii = seg(nb * 8);
    L.rho_in = seg(nc * 8);
    L.r2d = seg(nb * 8);
    L.r2f = seg(nb * 4);
    L.rhod = seg(nc * 8);
    L.rhof = seg(nc * 4);
    L.inv_mass = seg(nc * 8);
    L.inv_massf = seg(nc * 4);
    L.kA_d = seg(nc * 8);
    L.kA_f = seg(nc * 4);
    L.geo = seg(nb * 16);
    L.rhoe = seg(nb * 4);
    L.E = seg(nc * 8);
    L.Es = seg(nc * kAccSpreadBytes);  // IRE accumulator, one 256-byte segment per cell
    L.Eprev = seg(nc * 4);
    L.Ecur = seg(nc * kAccSpreadBytes);  // cell c at c * kCStride
    L.T = seg(nc * 8);
    L.sed = seg(nm * kMaxFreq * 8);
    const size_t rp = (size_t)tally_replicas();
    L.sed_q = seg(rp * nm * 2 * kMaxFreq * 8);
    L.inj_q = seg(rp * nm * 2 * 8);
    L.dir_q = seg(rp * nm * 2 * 8);
    L.freq = seg(kMaxFreq * 8);
    L.kabs = seg(kMaxFreq * 8);
    L.ksca = seg(kMaxFreq * 8);
    L.g = seg(kMaxFreq * 8);
    L.J = seg(kMaxFreq * 8);
    L.spec = seg(kMaxFreq * 8);
    L.dnu = seg(kMaxFreq * 8);
    L.src_cdf_d = seg(2 * kMaxFreq * 8);
    L.src_alias = seg(2 * kMaxFreq * 4);
    L.src_sum = seg(2 * 8);
    L.Lnode_d = seg(np2 * 8);
    L.Lnode_f = seg(np2 * 4);
    L.lnT = seg(np2 * 8);
    L.dalias = seg(nt * kMaxFreq * 4);
    L.dcdf_d = seg(nt * kMaxFreq * 8);
    L.dcdf_f = seg(nt * kMaxFreq * 4);
    L.nguide = seg(kGuide * 2);
    L.nmeta = seg(2 * 4);
    L.counters = seg(16 * 8);
    L.energies = seg(8 * 8);
    L.queue = seg(2 * 8);
    L.status = seg(4);
    L.diag = seg(16 * 4);
    L.seedw = seg(8);
    L.total = o;
    return L;
  }

  // Replicas of the batch tallies: enough that about 4096 model slots take
  // the escapes of a few models (a power of two, at most 64; 1 for a single
  // model, whose tallies live in shared memory).
  int tally_replicas() const {
    if (n_models <= 1) return 1;
    int r = 1;
    while (r < 64 && (long long)r * 2 * n_models <= 4096) r *= 2;
    return r;
  }

  int source_mask_single() const { return (has_ext ? 1 : 0) | (L_point > 0.0 ? 2 : 0); }

  // Per-model descriptors from the host inputs (work offsets in source slots).
  void fill_desc() {
    unsigned long long slot = 0;
    for (int m = 0; m < n_models; ++m) {
      ModelDesc &d = desc[m];
      int mask = kind.empty() || kind[m] == 0 ? source_mask_single() : kind[m];
      if (!has_ext) mask &= ~1;
      if (!(L_point > 0.0)) mask &= ~2;
      d.src_mask = mask;
      d.n_src = (mask & 1) + ((mask >> 1) & 1);
      const double *r = radii.data() + d.bnd_off;
      d.R = r[d.n_cells];
      d.point_cell = (r[0] > 0.0) ? -1 : 0;
      int n64 = 0;
      if (prec == PREC_MIXED && fp64_radius > 0.0)
        while (n64 < d.n_cells && r[n64 + 1] < fp64_radius * d.R) ++n64;
      d.n_fp64 = n64;
      d.pkg_off = slot;
      slot += (unsigned long long)d.n_src;
      d.L[0] = d.L[1] = 0.0;
    }
  }

  unsigned long long total_slots() const {
    unsigned long long s = 0;
    for (const auto &d : desc) s += (unsigned long long)d.n_src;
    return s;
  }

  int ensure_device() {
    if (sm_count == 0) {
      int dev = 0, count = 0;
      cudaError_t e = cudaGetDeviceCount(&count);
      if (e != cudaSuccess || count == 0)
        return fail(DIES_ECUDA, "no CUDA device available (%s)", cudaGetErrorString(e));
      DIES_CUDA(cudaGetDevice(&dev));
      DIES_CUDA(cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev));
    }
    if (!events_ready) {
      for (auto &e : ev) DIES_CUDA(cudaEventCreate(&e));
      events_ready = true;
    }
    const Layout L = layout();
    if (!ws || L.total > ws_bytes) {
      if (ws && !ws_owned) return fail(DIES_ENOMEM, "workspace of %zu bytes is smaller than the %zu needed", ws_bytes, L.total);
      if (ws_owned && ws) {
        cudaFree(ws);
        ws = nullptr;
      }
      void *p = nullptr;
      cudaError_t e = cudaMalloc(&p, L.total);
      if (e != cudaSuccess) return fail(DIES_ENOMEM, "cudaMalloc(%zu) failed: %s", L.total, cudaGetErrorString(e));
      ws = (unsigned char *)p;
      ws_bytes = L.total;
      ws_owned = true;
      tables_valid = false;
    }
    lay = L;
    return DIES_OK;
  }

  int upload(size_t off, const void *src, size_t bytes) {
    if (bytes == 0) return DIES_OK;
    DIES_CUDA(cudaMemcpyAsync(ws + off, src, bytes, cudaMemcpyHostToDevice, stream));
    return DIES_OK;
  }

  bool kA_weighting() const { return kA_rho || k_A != 1.0; }

  // Absorption free-path factor per shell (Sect. 2.2.2): the constant k_A,
  // or linear in log density from kA_lo at each model's lowest positive
  // shell density to kA_hi at its highest (empty shells: kA_lo).
  void kA_cells(std::vector<double> &out) const {
    out.assign((size_t)n_cells, k_A);
    if (!kA_rho) return;
    for (int m = 0; m < n_models; ++m) {
      const int c0 = desc[m].cell_off, n = desc[m].n_cells;
      double lmin = 0.0, lmax = 0.0;
      bool any = false;
      for (int i = 0; i < n; ++i) {
        const double r = rho[c0 + i];
        if (!(r > 0.0)) continue;
        const double l = std::log(r);
        if (!any || l < lmin) lmin = l;
        if (!any || l > lmax) lmax = l;
        any = true;
      }
      for (int i = 0; i < n; ++i) {
        const double r = rho[c0 + i];
        if (!(r > 0.0)) out[c0 + i] = kA_lo;
        else if (!(lmax > lmin)) out[c0 + i] = kA_hi;
        else out[c0 + i] = kA_hi + (kA_lo - kA_hi) * (lmax - std::log(r)) / (lmax - lmin);
      }
    }
  }

  int build_tables() {
    Range r("dies: upload + table build");
    fill_desc();
    int rc;
    if ((rc = upload(lay.desc, desc.data(), desc.size() * sizeof(ModelDesc)))) return rc;
    {
      std::vector<double> kd;
      kA_cells(kd);
      std::vector<float> kf(kd.begin(), kd.end());
      if ((rc = upload(lay.kA_d, kd.data(), kd.size() * 8))) return rc;
      if ((rc = upload(lay.kA_f, kf.data(), kf.size() * 4))) return rc;
    }
    if ((rc = upload(lay.radii, radii.data(), radii.size() * 8))) return rc;
    if ((rc = upload(lay.rho_in, rho.data(), rho.size() * 8))) return rc;
    std::vector<double> pad(6 * kMaxFreq, 0.0);
    for (int k = 0; k < F; ++k) {
      pad[0 * kMaxFreq + k] = freq[k];
      pad[1 * kMaxFreq + k] = kabs[k];
      pad[2 * kMaxFreq + k] = ksca[k];
      pad[3 * kMaxFreq + k] = g[k];
      pad[4 * kMaxFreq + k] = has_ext ? J[k] : 0.0;
      pad[5 * kMaxFreq + k] = (L_point > 0.0) ? spec[k] : 0.0;
    }
    const size_t offs[6] = {lay.freq, lay.kabs, lay.ksca, lay.g, lay.J, lay.spec};
    for (int i = 0; i < 6; ++i)
      if ((rc = upload(offs[i], pad.data() + i * kMaxFreq, kMaxFreq * 8))) return rc;
    DIES_CUDA(cudaEventRecord(ev[5], stream));
    DIES_CUDA(launch_freq_tables(stream, F, at<double>(lay.freq), has_ext ? at<double>(lay.J) : nullptr,
                                 (L_point > 0.0) ? at<double>(lay.spec) : nullptr, at<double>(lay.dnu),
                                 at<double>(lay.src_cdf_d), at<uint32_t>(lay.src_alias), at<double>(lay.src_sum)));
    DIES_CUDA(launch_node_tables(stream, F, n_tnodes, next_pow2(n_tnodes), T_min, T_max, at<double>(lay.freq),
                                 at<double>(lay.kabs), at<double>(lay.dnu), at<double>(lay.Lnode_d),
                                 at<float>(lay.Lnode_f), at<double>(lay.lnT), at<uint32_t>(lay.dalias),
                                 at<double>(lay.dcdf_d), at<float>(lay.dcdf_f), at<uint16_t>(lay.nguide),
                                 at<int>(lay.nmeta)));
    DIES_CUDA(launch_geometry(stream, n_models, at<ModelDesc>(lay.desc), n_cells, n_cells + n_models,
                              at<double>(lay.radii), at<double>(lay.rho_in), length_unit_cm, at<double>(lay.src_sum),
                              L_point, at<double>(lay.r2d), at<float>(lay.r2f), at<double>(lay.rhod),
                              at<float>(lay.rhof), at<double>(lay.inv_mass), at<float>(lay.inv_massf),
                              at<float4>(lay.geo), at<float>(lay.rhoe)));
    tables_valid = true;
    return DIES_OK;
  }

  TransportParams params(int mode, uint64_t n, uint64_t seed) const {
    TransportParams P{};
    P.desc = at<ModelDesc>(lay.desc);
    P.n_models = n_models;
    P.F = F;
    P.r2f = at<float>(lay.r2f);
    P.r2d = at<double>(lay.r2d);
    P.rhof = at<float>(lay.rhof);
    P.rhod = at<double>(lay.rhod);
    P.inv_mass = at<double>(lay.inv_mass);
    P.inv_massf = at<float>(lay.inv_massf);
    P.geo = at<float4>(lay.geo);
    P.rhoe = at<float>(lay.rhoe);
    P.sed_q = at<unsigned long long>(lay.sed_q);
    P.inj_q = at<unsigned long long>(lay.inj_q);
    P.dir_q = at<unsigned long long>(lay.dir_q);
    P.rep = tally_replicas();
    // IRE runs add absorbed energies into the spread accumulator (E is
    // filled from it by the finalize kernel); the frozen passes into E
    const bool ire = (mode == MODE_IRE);
    P.E = at<double>(ire ? lay.Es : lay.E);
    P.e_stride = ire ? kEStride : 1;
    P.Eprev = at<float>(lay.Eprev);
    P.Ecur = at<float>(lay.Ecur);
    P.c_stride = kCStride;
    P.sgeo_n = (mode == MODE_IRE) ? sgeo_n : 0;
    P.sed = at<double>(lay.sed);
    P.kabs_d = at<double>(lay.kabs);
    P.ksca_d = at<double>(lay.ksca);
    P.g_d = at<double>(lay.g);
    P.src_cdf_d = at<double>(lay.src_cdf_d);
    P.Lnode_d = at<double>(lay.Lnode_d);
    P.Lnode_f = at<float>(lay.Lnode_f);
    P.dalias = at<uint32_t>(lay.dalias);
    P.src_alias = at<uint32_t>(lay.src_alias);
    P.nguide = at<uint16_t>(lay.nguide);
    P.nmeta = at<int>(lay.nmeta);
    P.dcdf_d = at<double>(lay.dcdf_d);
    P.dcdf_f = at<float>(lay.dcdf_f);
    P.remit_cdf = remit_table;
    P.refill_div = (unsigned)refill_div;
    P.pool = (pkgs_per_thread == 2 && mode == MODE_IRE) ? 1 : 0;
    P.n_tnodes = n_tnodes;
    P.n_tnodes_pow2 = next_pow2(n_tnodes);
    P.n_per_source = n;
    P.pkg_begin = 0;
    P.pkg_len = n;
    P.total = total_slots() * n;
    P.seed = seed;
    P.queue = at<unsigned long long>(lay.queue);
    P.counters = at<unsigned long long>(lay.counters);
    P.energies = at<double>(lay.energies);
    P.status = at<uint32_t>(lay.status);
    P.diag = at<uint32_t>(lay.diag);
    P.k_bg = k_bg;
    P.ffi = ffi;
    P.mode = mode;
    P.max_events = 100000000ULL;
    P.time_budget_ns = (unsigned long long)(time_budget_s * 1e9);
    P.inv_n = (float)(0x1p64 / (double)n);
    P.inv_nd = 1.0 / (double)n;
    P.k_bg_f = (float)k_bg;
    P.g_E = g_E;
    P.g_S = g_S;
    P.k_S = k_S;
    P.scat_w = scat_w;
    P.kA_d = kA_weighting() ? at<double>(lay.kA_d) : nullptr;
    P.kA_f = kA_weighting() ? at<float>(lay.kA_f) : nullptr;
    P.kA_void = kA_rho ? kA_lo : k_A;
    P.g_E_f = (float)g_E;
    P.g_S_f = (float)g_S;
    P.k_S_f = (float)k_S;
    P.kA_void_f = (float)P.kA_void;
    P.remit_random = remit_random;
    P.radii_d = at<double>(lay.radii);
    P.kbg_plain = (k_bg == 0.5);
    P.r64 = (prec == PREC_MIXED && fp64_radius > 0.0);
    P.batch_min = rare_batch;
    P.inner = inner;
    P.agg = agg;
    return P;
  }

  // Grid of the next launch, and whether it stages the geometry in shared
  // memory: only for one model without FP64 crossings or package pools, and
  // only where the staged records cost no resident CTA.
  int grid_for(int prec_, int mode, int *grid) {
    int bps = blocks_per_sm;
    int occ = 0;
    const bool r64 = (prec_ == PREC_MIXED && fp64_radius > 0.0);
    const bool pool = pkgs_per_thread == 2;
    sgeo_n = 0;
    const bool plain = plain_weighting(params(mode, 1, 0));  // the kernel variant the launch will pick
    DIES_CUDA(transport_occupancy(prec_, mode, block, next_pow2(n_tnodes), r64, ffi != 0, n_models > 1, pool, plain,
                                  agg != 0, 0, &occ));
    if (occ < 1) return fail(DIES_ECUDA, "transport kernel cannot be resident with block size %d", block);
    if (bps <= 0 || bps > occ) bps = occ;
    if (stage_geo && mode == MODE_IRE && n_models == 1 && prec_ != PREC_FP64 && !r64 && !(pool && ffi == 0)) {
      int occ_s = 0;
      // a refusal here (staged records beyond the shared-memory limit) only means: no staging
      if (transport_occupancy(prec_, mode, block, next_pow2(n_tnodes), false, ffi != 0, false, pool, plain,
                              agg != 0, n_cells + 1, &occ_s) != cudaSuccess) {
        cudaGetLastError();
        occ_s = 0;
      }
      if (occ_s >= bps) sgeo_n = n_cells + 1;
    }
    *grid = sm_count * bps;
    last_grid = (uint32_t)*grid;
    last_block = (uint32_t)block;
    last_variant = 0;
    if (mode == MODE_IRE && prec_ != PREC_FP64) {
      if (plain) last_variant |= DIES_VARIANT_PLAIN_WEIGHTING;
      if (sgeo_n > 0) last_variant |= DIES_VARIANT_STAGED_GEOMETRY;
      if (pool && ffi == 0) last_variant |= DIES_VARIANT_PACKAGE_POOL;
      if (r64) last_variant |= DIES_VARIANT_FP64_CROSSINGS;
    }
    return DIES_OK;
  }

  int reset_accumulators(bool resume = false) { return reset_accumulators_on(stream, resume); }

  // the package range of this run ([first, first + count) of n), checked
  int take_range(uint64_t n, uint64_t *first, uint64_t *count, bool *resume) {
    *first = 0;
    *count = n;
    *resume = false;
    if (!range_set) return DIES_OK;
    range_set = false;  // applies to one run
    if (range_count == 0 || range_first > n || range_count > n - range_first)
      return fail(DIES_EINVAL, "package range [%llu, %llu) does not lie in [0, %llu)",
                  (unsigned long long)range_first, (unsigned long long)(range_first + range_count),
                  (unsigned long long)n);
    if (range_resume && !has_result) return fail(DIES_ESTATE, "resume needs a previous run on this handle");
    *first = range_first;
    *count = range_count;
    *resume = range_resume;
    return DIES_OK;
  }
  // resume: keep absorbed energies, tallies, counters and energy sums of the
  // previous run; only the work counter, status and diagnostics restart
  int reset_accumulators_on(cudaStream_t st, bool resume = false) {
    if (resume) {
      DIES_CUDA(cudaMemsetAsync(ws + lay.queue, 0, 2 * 8, st));
      DIES_CUDA(cudaMemsetAsync(ws + lay.status, 0, 4, st));
      DIES_CUDA(cudaMemsetAsync(ws + lay.diag, 0, 16 * 4, st));
      return DIES_OK;
    }
    DIES_CUDA(cudaMemsetAsync(ws + lay.E, 0, (size_t)n_cells * 8, st));
    DIES_CUDA(cudaMemsetAsync(ws + lay.Es, 0, (size_t)n_cells * kAccSpreadBytes, st));
    DIES_CUDA(cudaMemsetAsync(ws + lay.Eprev, 0, (size_t)n_cells * 4, st));
    DIES_CUDA(cudaMemsetAsync(ws + lay.Ecur, 0, (size_t)n_cells * kAccSpreadBytes, st));
    DIES_CUDA(cudaMemsetAsync(ws + lay.sed, 0, (size_t)n_models * kMaxFreq * 8, st));
    const size_t rp = (size_t)tally_replicas();
    DIES_CUDA(cudaMemsetAsync(ws + lay.sed_q, 0, rp * n_models * 2 * kMaxFreq * 8, st));
    DIES_CUDA(cudaMemsetAsync(ws + lay.inj_q, 0, rp * n_models * 2 * 8, st));
    DIES_CUDA(cudaMemsetAsync(ws + lay.dir_q, 0, rp * n_models * 2 * 8, st));
    DIES_CUDA(cudaMemsetAsync(ws + lay.counters, 0, 16 * 8 + 0, st));
    DIES_CUDA(cudaMemsetAsync(ws + lay.energies, 0, 8 * 8, st));
    DIES_CUDA(cudaMemsetAsync(ws + lay.queue, 0, 2 * 8, st));
    DIES_CUDA(cudaMemsetAsync(ws + lay.status, 0, 4, st));
    DIES_CUDA(cudaMemsetAsync(ws + lay.diag, 0, 16 * 4, st));
    return DIES_OK;
  }

  int check_ready() const {
    if (!has_dust) return fail(DIES_ESTATE, "dust not set (dies_set_dust)");
    if (!has_sources) return fail(DIES_ESTATE, "sources not set (dies_set_sources)");
    return DIES_OK;
  }

  // Enqueue a full IRE run.
  int enqueue_run(uint64_t n, uint64_t seed) {
    int rc;
    if ((rc = check_ready())) return rc;
    if (n == 0) return fail(DIES_EINVAL, "n_packages must be >= 1");
    const bool ranged = range_set;
    uint64_t first, count;
    bool resume;
    if ((rc = take_range(n, &first, &count, &resume))) return rc;
    if ((rc = ensure_device())) return rc;
    launches_at_start = g_launches.load();
    DIES_CUDA(cudaEventRecord(ev[0], stream));
    table_built_this_run = false;
    if (!tables_valid) {
      if ((rc = build_tables())) return rc;
      table_built_this_run = true;
    }
    DIES_CUDA(cudaEventRecord(ev[1], stream));
    int grid;
    if ((rc = grid_for(prec, MODE_IRE, &grid))) return rc;
    if (use_graph && !ranged) {
      if ((rc = replay_graph(n, seed, grid))) return rc;
    } else {
      if ((rc = enqueue_body(stream, n, seed, grid, nullptr, first, count, resume))) return rc;
    }
    DIES_CUDA(cudaEventRecord(ev[4], stream));
    has_result = true;
    stats_pending = true;
    static_pending = false;
    e_in_fp32_counters = (prec == PREC_FP32);
    return DIES_OK;
  }

  // The per-run device work after the table build: accumulator reset, the
  // transport launch(es), tallies and temperatures, on stream st.  With
  // seed_dev set (graph capture) the kernels read the seed from there and
  // the timing events are recorded as graph nodes.
  int enqueue_body(cudaStream_t st, uint64_t n, uint64_t seed, int grid, const unsigned long long *seed_dev,
                   uint64_t first = 0, uint64_t count = 0, bool resume = false) {
    Range r("dies: enqueue transport + temperatures");
    int rc;
    if (count == 0) count = n;
    const unsigned rec_flags = seed_dev ? cudaEventRecordExternal : cudaEventRecordDefault;
    if ((rc = reset_accumulators_on(st, resume))) return rc;
    TransportParams P = params(MODE_IRE, n, seed);
    P.seed_dev = seed_dev;
    DIES_CUDA(cudaEventRecordWithFlags(ev[2], st, rec_flags));
    // packages [first, first + count) of each source, in N_B sequential batches in the FP32 form
    const int nb = (prec == PREC_FP32) ? n_batches : 1;
    const uint64_t per = (count + nb - 1) / nb;
    for (int b = 0; b < nb; ++b) {
      const uint64_t begin = first + (uint64_t)b * per;
      if (begin >= first + count) break;
      const uint64_t len = (begin + per <= first + count) ? per : first + count - begin;
      P.pkg_begin = begin;
      P.pkg_len = len;
      P.total = total_slots() * len;
      P.queue = at<unsigned long long>(lay.queue) + (b & 1);
      if (b > 0) DIES_CUDA(cudaMemsetAsync(P.queue, 0, 8, st));
      DIES_CUDA(launch_transport(prec, MODE_IRE, false, P, grid, block, st));
      if (prec == PREC_FP32) DIES_CUDA(launch_merge(st, n_cells, at<float>(lay.Eprev), at<float>(lay.Ecur)));
    }
    DIES_CUDA(cudaEventRecordWithFlags(ev[3], st, rec_flags));
    // the FP32 forms' tally kernel adds the (cumulative) fixed-point injection
    // and direct-escape tallies: their energy sums restart from zero
    if (prec != PREC_FP64 && resume) {
      DIES_CUDA(cudaMemsetAsync(ws + lay.energies + EN_INJECTED * 8, 0, 8, st));
      DIES_CUDA(cudaMemsetAsync(ws + lay.energies + EN_DIRECT * 8, 0, 8, st));
    }
    if (prec != PREC_FP64)
      DIES_CUDA(launch_tally(st, n_models, at<ModelDesc>(lay.desc), n, at<unsigned long long>(lay.sed_q),
                             at<unsigned long long>(lay.inj_q), at<unsigned long long>(lay.dir_q), at<double>(lay.sed),
                             at<double>(lay.energies), tally_replicas()));
    DIES_CUDA(launch_finalize(st, n_cells, at<double>(lay.Es), at<float>(lay.Eprev), at<float>(lay.Ecur),
                              prec == PREC_FP32, at<double>(lay.inv_mass), at<double>(lay.Lnode_d),
                              at<double>(lay.lnT), n_tnodes, at<double>(lay.T), at<double>(lay.E)));
    return DIES_OK;
  }

  // Graph mode: capture enqueue_body once per configuration (on a private
  // stream), then replay it on the handle's stream; the seed travels through
  // a pinned host word that the graph copies to the device first.
  int replay_graph(uint64_t n, uint64_t seed, int grid) {
    GraphKey k;
    std::memset(&k, 0, sizeof k);
    k.P = params(MODE_IRE, n, 0);
    k.n = n;
    k.prec = prec;
    k.n_batches = n_batches;
    k.grid = grid;
    k.block = block;
    k.n_cells = n_cells;
    k.n_models = n_models;
    k.n_tnodes = n_tnodes;
    if (!graph_valid || std::memcmp(&k, &gkey, sizeof k) != 0) {
      drop_graph();
      if (!cap_stream) DIES_CUDA(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
      if (!seed_host) {
        void *h = nullptr;
        cudaError_t e = cudaHostAlloc(&h, 8, cudaHostAllocDefault);
        if (e != cudaSuccess) return fail(DIES_ENOMEM, "pinned seed word: %s", cudaGetErrorString(e));
        seed_host = static_cast<unsigned long long *>(h);
      }
      // the capture stream must not run ahead of work already on the handle's stream
      DIES_CUDA(cudaStreamSynchronize(stream));
      const unsigned long long before = g_launches.load();
      DIES_CUDA(cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeRelaxed));
      const unsigned long long *seed_dev = at<unsigned long long>(lay.seedw);
      cudaError_t e = cudaMemcpyAsync(ws + lay.seedw, seed_host, 8, cudaMemcpyHostToDevice, cap_stream);
      int rc = (e == cudaSuccess) ? enqueue_body(cap_stream, n, 0, grid, seed_dev)
                                  : fail(DIES_ECUDA, "capture: %s", cudaGetErrorString(e));
      cudaGraph_t g = nullptr;
      const cudaError_t ee = cudaStreamEndCapture(cap_stream, &g);
      graph_kernels = g_launches.load() - before;
      g_launches.fetch_sub(graph_kernels);  // captured, not launched
      if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (ee != cudaSuccess) return fail(DIES_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ee));
      graph = g;
      e = cudaGraphInstantiate(&gexec, graph, 0);
      if (e != cudaSuccess) {
        drop_graph();
        return fail(DIES_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
      }
      gkey = k;
      graph_valid = true;
    }
    // the previous replay may not have copied its seed yet
    DIES_CUDA(cudaStreamSynchronize(stream));
    *seed_host = seed;
    DIES_CUDA(cudaGraphLaunch(gexec, stream));
    launch_counter_add((unsigned)graph_kernels);
    return DIES_OK;
  }

  // Wait for the stream and collect the counters of the last run (of the
  // last static frozen pass if that came last: its words sit in the static
  // scratch, and only host stack memory receives them).
  int collect() {
    if (!has_result) return fail(DIES_ESTATE, "no run has completed on this handle");
    Range r("dies: wait + read-back");
    DIES_CUDA(cudaStreamSynchronize(stream));
    if (!stats_pending) {
      if (stats.status_word & STATUS_TIMEOUT) return DIES_ETIMEOUT;
      return (stats.status_word & (STATUS_RANGE | STATUS_BOUNDS)) ? DIES_ERANGE : DIES_OK;
    }
    const bool st = static_pending;
    unsigned long long cnt[16];
    double en[8];
    uint32_t status = 0;
    double sed_stat[kMaxFreq];
    std::vector<double> sed(st ? 0 : (size_t)n_models * kMaxFreq);
    DIES_CUDA(cudaMemcpy(cnt, st ? static_counters : ws + lay.counters, sizeof cnt, cudaMemcpyDeviceToHost));
    DIES_CUDA(cudaMemcpy(en, st ? static_energies : ws + lay.energies, sizeof en, cudaMemcpyDeviceToHost));
    DIES_CUDA(cudaMemcpy(&status, st ? static_status : ws + lay.status, 4, cudaMemcpyDeviceToHost));
    uint32_t diag[16];
    DIES_CUDA(cudaMemcpy(diag, st ? static_diag : ws + lay.diag, sizeof diag, cudaMemcpyDeviceToHost));
    if (st) DIES_CUDA(cudaMemcpy(sed_stat, static_sed, sizeof sed_stat, cudaMemcpyDeviceToHost));
    else DIES_CUDA(cudaMemcpy(sed.data(), ws + lay.sed, sed.size() * 8, cudaMemcpyDeviceToHost));
    dies_stats s{};
    s.injected = cnt[CNT_INJECTED];
    s.escaped = cnt[CNT_ESCAPED];
    s.absorbed = cnt[CNT_ABSORB];
    s.scattered = cnt[CNT_SCATTER];
    s.crossed = cnt[CNT_CROSS];
    s.killed_weight = cnt[CNT_KILL_WEIGHT];
    s.killed_cap = cnt[CNT_KILL_CAP];
    s.clamp_hi = cnt[CNT_CLAMP_HI];
    s.forced = cnt[CNT_FORCED];
    s.E_injected = en[EN_INJECTED];
    s.E_lost = en[EN_LOST];
    s.E_direct = en[EN_DIRECT];
    double esc = 0.0;
    if (st) {
      for (int k = 0; k < kMaxFreq; ++k) esc += sed_stat[k];
    } else {
      for (double v : sed) esc += v;
    }
    s.E_escaped = esc;
    float ms = 0.0f;
    if (!st) {  // the static pass records no timing events
      if (cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess) s.table_ms = table_built_this_run ? ms : 0.0;
      if (table_built_this_run && cudaEventElapsedTime(&ms, ev[0], ev[5]) == cudaSuccess) s.upload_ms = ms;
      if (cudaEventElapsedTime(&ms, ev[1], ev[4]) == cudaSuccess) s.kernel_ms = ms;
      if (cudaEventElapsedTime(&ms, ev[2], ev[3]) == cudaSuccess) s.transport_ms = ms;
    }
    s.status_word = status;
    for (int i = 0; i < 16; ++i) s.diag[i] = diag[i];
    s.launches = (uint32_t)(g_launches.load() - launches_at_start);
    if (!st) {
      s.grid = last_grid;
      s.block = last_block;
      s.variant = last_variant;
    }
    stats = s;
    stats_pending = false;
    static_pending = false;
    if (status & STATUS_TIMEOUT) return fail(DIES_ETIMEOUT, "transport kernel stopped at its time budget");
    if (status & STATUS_RANGE)
      return fail(DIES_ERANGE, "an absorbed-energy counter of the all-FP32 form left the FP32 range "
                               "(luminosity above ~1e38 erg/s): use DIES_PREC_MIXED");
    if (status & STATUS_BOUNDS)
      return fail(DIES_ERANGE, "device bounds check failed (check build; status 0x%x): an index left its table",
                  status);
    return DIES_OK;
  }

  int frozen(const double *T_frozen, uint64_t n, uint64_t seed, int flags, uint32_t *ev_out, uint64_t *hash_out) {
    Range r("dies: frozen pass");
    int rc;
    if ((rc = check_ready())) return rc;
    if (n == 0) return fail(DIES_EINVAL, "n_packages must be >= 1");
    if (!T_frozen) return fail(DIES_EINVAL, "T_frozen is NULL");
    for (int i = 0; i < n_cells; ++i)
      if (!(std::isfinite(T_frozen[i]) && T_frozen[i] > 0.0))
        return fail(DIES_EINVAL, "T_frozen[%d] must be finite and > 0", i);
    const bool in_form = (flags & DIES_FROZEN_FORM) != 0;
    const int base = flags & ~DIES_FROZEN_FORM;
    if (base != DIES_FROZEN_REEMIT && base != DIES_FROZEN_ABSORB_TERMINAL)
      return fail(DIES_EINVAL, "unknown frozen flags %d", flags);
    if (in_form && base != DIES_FROZEN_ABSORB_TERMINAL)
      return fail(DIES_EINVAL, "DIES_FROZEN_FORM needs DIES_FROZEN_ABSORB_TERMINAL");
    if (in_form && (ev_out || hash_out))
      return fail(DIES_EINVAL, "per-package records exist only in the FP64 form (n_events_out and path_hash_out must be NULL)");
    // the precision form of the pass: the handle's with DIES_FROZEN_FORM, else FP64
    const int fprec = in_form ? prec : PREC_FP64;
    uint64_t first, count;
    bool resume;
    if ((rc = take_range(n, &first, &count, &resume))) return rc;
    if ((rc = ensure_device())) return rc;
    launches_at_start = g_launches.load();
    DIES_CUDA(cudaEventRecord(ev[0], stream));
    table_built_this_run = false;
    if (!tables_valid) {
      if ((rc = build_tables())) return rc;
      table_built_this_run = true;
    }
    DIES_CUDA(cudaEventRecord(ev[1], stream));
    const unsigned long long rows = total_slots() * n;
    double *dT = nullptr, *dcdf = nullptr;
    uint32_t *dev = nullptr;
    unsigned long long *dhash = nullptr;
    auto release = [&]() {
      if (dT) cudaFree(dT);
      if (dcdf) cudaFree(dcdf);
      if (dev) cudaFree(dev);
      if (dhash) cudaFree(dhash);
    };
    cudaError_t e = cudaMalloc(&dT, (size_t)n_cells * 8);
    if (e == cudaSuccess) e = cudaMalloc(&dcdf, (size_t)n_cells * kMaxFreq * 8);
    if (e == cudaSuccess && ev_out) e = cudaMalloc(&dev, rows * 3 * 4);
    if (e == cudaSuccess && hash_out) e = cudaMalloc(&dhash, rows * 8);
    if (e != cudaSuccess) {
      release();
      return fail(DIES_ENOMEM, "frozen-pass buffers: %s", cudaGetErrorString(e));
    }
    rc = DIES_OK;
    do {
      if ((e = cudaMemcpyAsync(dT, T_frozen, (size_t)n_cells * 8, cudaMemcpyHostToDevice, stream))) break;
      if ((e = launch_frozen_cdf(stream, n_cells, F, at<double>(lay.freq), at<double>(lay.kabs), at<double>(lay.dnu),
                                 dT, dcdf)))
        break;
      if ((rc = reset_accumulators(resume))) break;
      const int mode = (base == DIES_FROZEN_ABSORB_TERMINAL) ? MODE_FROZEN_TERMINAL : MODE_FROZEN;
      int grid;
      if ((rc = grid_for(fprec, mode, &grid))) break;
      if ((e = cudaEventRecord(ev[2], stream))) break;
      TransportParams P = params(mode, n, seed);
      P.pkg_begin = first;
      P.pkg_len = count;
      P.total = total_slots() * count;
      P.cell_cdf = dcdf;
      P.rec_events = dev;
      P.rec_hash = dhash;
      if (fprec != PREC_MIXED) P.r64 = 0;
      if ((e = launch_transport(fprec, mode, ev_out || hash_out, P, grid, block, stream))) break;
      if ((e = cudaEventRecord(ev[3], stream))) break;
      // the FP32 forms keep their escape and injection tallies in fixed point
      if (fprec != PREC_FP64 && resume) {
        if ((e = cudaMemsetAsync(ws + lay.energies + EN_INJECTED * 8, 0, 8, stream))) break;
        if ((e = cudaMemsetAsync(ws + lay.energies + EN_DIRECT * 8, 0, 8, stream))) break;
      }
      if (fprec != PREC_FP64 &&
          (e = launch_tally(stream, n_models, at<ModelDesc>(lay.desc), n, at<unsigned long long>(lay.sed_q),
                            at<unsigned long long>(lay.inj_q), at<unsigned long long>(lay.dir_q), at<double>(lay.sed),
                            at<double>(lay.energies), tally_replicas())))
        break;
      if ((e = cudaMemcpyAsync(ws + lay.T, dT, (size_t)n_cells * 8, cudaMemcpyDeviceToDevice, stream))) break;
      if ((e = cudaEventRecord(ev[4], stream))) break;
      has_result = true;
      stats_pending = true;
      static_pending = false;
      e_in_fp32_counters = false;  // every frozen pass tallies in the FP64 accumulator
      if ((rc = collect())) break;
      if (ev_out && (e = cudaMemcpy(ev_out, dev, rows * 3 * 4, cudaMemcpyDeviceToHost))) break;
      if (hash_out && (e = cudaMemcpy(hash_out, dhash, rows * 8, cudaMemcpyDeviceToHost))) break;
    } while (0);
    release();
    if (e != cudaSuccess) return fail(DIES_ECUDA, "frozen pass: %s", cudaGetErrorString(e));
    return rc;
  }

  int get_cells(size_t off, double *out, int n) {
    if (!out) return fail(DIES_EINVAL, "output pointer is NULL");
    if (n != n_cells) return fail(DIES_EINVAL, "expected %d shells, got %d", n_cells, n);
    int rc = collect();
    if (rc && rc != DIES_ETIMEOUT && rc != DIES_ERANGE) return rc;
    DIES_CUDA(cudaMemcpy(out, ws + off, (size_t)n * 8, cudaMemcpyDeviceToHost));
    return rc;
  }

  int get_sed(double *out, int n) {
    if (!out) return fail(DIES_EINVAL, "output pointer is NULL");
    if (n != n_models * F) return fail(DIES_EINVAL, "expected %d values, got %d", n_models * F, n);
    int rc = collect();
    if (rc && rc != DIES_ETIMEOUT && rc != DIES_ERANGE) return rc;
    std::vector<double> tmp((size_t)n_models * kMaxFreq);
    DIES_CUDA(cudaMemcpy(tmp.data(), ws + lay.sed, tmp.size() * 8, cudaMemcpyDeviceToHost));
    for (int m = 0; m < n_models; ++m)
      for (int k = 0; k < F; ++k) out[(size_t)m * F + k] = tmp[(size_t)m * kMaxFreq + k];
    return rc;
  }

  // -------------------------------------------------------------- setters
  int set_dust(const double *nu, int n, const double *ka, const double *ks, const double *gg) {
    if (!nu || !ka || !ks || !gg) return fail(DIES_EINVAL, "dust arrays must not be NULL");
    if (n < 2 || n > DIES_MAX_FREQ) return fail(DIES_EINVAL, "n_freq must be in [2, %d], got %d", DIES_MAX_FREQ, n);
    for (int k = 0; k < n; ++k) {
      if (!(std::isfinite(nu[k]) && nu[k] > 0.0)) return fail(DIES_EINVAL, "freq_hz[%d] must be finite and > 0", k);
      if (k > 0 && !(nu[k] > nu[k - 1])) return fail(DIES_EINVAL, "freq_hz must be strictly increasing");
      if (!(std::isfinite(ka[k]) && ka[k] >= 0.0)) return fail(DIES_EINVAL, "kappa_abs[%d] must be finite and >= 0", k);
      if (!(std::isfinite(ks[k]) && ks[k] >= 0.0)) return fail(DIES_EINVAL, "kappa_sca[%d] must be finite and >= 0", k);
      if (!(std::fabs(gg[k]) < 1.0)) return fail(DIES_EINVAL, "g[%d] must lie in (-1, 1)", k);
    }
    if (has_sources && n != F) has_sources = false;  // source spectra no longer match
    F = n;
    freq.assign(nu, nu + n);
    kabs.assign(ka, ka + n);
    ksca.assign(ks, ks + n);
    g.assign(gg, gg + n);
    has_dust = true;
    tables_valid = false;
    return DIES_OK;
  }

  int set_sources(const double *Jx, double Lp, const double *sp) {
    if (!has_dust) return fail(DIES_ESTATE, "call dies_set_dust before dies_set_sources");
    if (!std::isfinite(Lp) || Lp < 0.0) return fail(DIES_EINVAL, "L_point must be finite and >= 0");
    if (!Jx && !(Lp > 0.0)) return fail(DIES_EINVAL, "at least one source (J_ext or L_point > 0) is required");
    if (Lp > 0.0 && !sp) return fail(DIES_EINVAL, "point_spectrum is required when L_point > 0");
    double sj = 0.0, ss = 0.0;
    if (Jx) {
      if (!finite_nonneg(Jx, F)) return fail(DIES_EINVAL, "J_ext must be finite and >= 0");
      for (int k = 0; k < F; ++k) sj += Jx[k];
      if (!(sj > 0.0)) return fail(DIES_EINVAL, "J_ext is zero at every frequency");
    }
    if (Lp > 0.0) {
      if (!finite_nonneg(sp, F)) return fail(DIES_EINVAL, "point_spectrum must be finite and >= 0");
      for (int k = 0; k < F; ++k) ss += sp[k];
      if (!(ss > 0.0)) return fail(DIES_EINVAL, "point_spectrum is zero at every frequency");
    }
    has_ext = Jx != nullptr;
    J.assign(Jx ? Jx : sp, (Jx ? Jx : sp) + (Jx ? F : 0));
    L_point = Lp;
    spec.assign(sp ? sp : Jx, (sp ? sp : Jx) + ((Lp > 0.0) ? F : 0));
    has_sources = true;
    tables_valid = false;
    return DIES_OK;
  }
};

}  // namespace dies

using dies::fail;
using dies::Problem;

struct dies_model {
  Problem p;
};
struct dies_batch {
  Problem p;
};

namespace {

int check_geometry(const double *radii, int n_radii, const double *rho, int n_shells, double lu) {
  if (!radii || !rho) return fail(DIES_EINVAL, "radii and densities must not be NULL");
  if (n_shells < 1 || n_shells > DIES_MAX_SHELLS)
    return fail(DIES_EINVAL, "n_shells must be in [1, %d], got %d", DIES_MAX_SHELLS, n_shells);
  if (n_radii != n_shells + 1) return fail(DIES_EINVAL, "n_radii must equal n_shells + 1");
  if (!(std::isfinite(radii[0]) && radii[0] >= 0.0)) return fail(DIES_EINVAL, "radii[0] must be finite and >= 0");
  for (int i = 0; i < n_shells; ++i) {
    if (!(std::isfinite(radii[i + 1]) && radii[i + 1] > radii[i]))
      return fail(DIES_EINVAL, "radii must be finite and strictly increasing (index %d)", i + 1);
    if (!(std::isfinite(rho[i]) && rho[i] >= 0.0))
      return fail(DIES_EINVAL, "densities[%d] must be finite and >= 0", i);
  }
  if (!(std::isfinite(lu) && lu > 0.0)) return fail(DIES_EINVAL, "length_unit_cm must be finite and > 0");
  return DIES_OK;
}

}  // namespace

extern "C" {

int dies_create_model(const double *radii, int n_radii, const double *densities, int n_shells,
                      double length_unit_cm, dies_model **out) {
  if (!out) return fail(DIES_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = check_geometry(radii, n_radii, densities, n_shells, length_unit_cm);
  if (rc) return rc;
  dies_model *m = new (std::nothrow) dies_model();
  if (!m) return fail(DIES_ENOMEM, "host allocation failed");
  Problem &p = m->p;
  p.n_models = 1;
  p.n_cells = n_shells;
  p.radii.assign(radii, radii + n_radii);
  p.rho.assign(densities, densities + n_shells);
  p.length_unit_cm = length_unit_cm;
  p.desc.resize(1);
  p.desc[0] = dies::ModelDesc{};
  p.desc[0].cell_off = 0;
  p.desc[0].bnd_off = 0;
  p.desc[0].n_cells = n_shells;
  *out = m;
  return DIES_OK;
}

int dies_set_dust(dies_model *m, const double *freq_hz, int n_freq, const double *kappa_abs,
                  const double *kappa_sca, const double *g) {
  if (!m) return fail(DIES_EINVAL, "model is NULL");
  return m->p.set_dust(freq_hz, n_freq, kappa_abs, kappa_sca, g);
}

int dies_set_sources(dies_model *m, const double *J_ext, double L_point, const double *point_spectrum) {
  if (!m) return fail(DIES_EINVAL, "model is NULL");
  return m->p.set_sources(J_ext, L_point, point_spectrum);
}

int dies_set_weighting(dies_model *m, double k_bg, int ffi) {
  if (!m) return fail(DIES_EINVAL, "model is NULL");
  if (!(k_bg > 0.0 && k_bg <= 1.0)) return fail(DIES_EINVAL, "k_bg must lie in (0, 1]");
  if (ffi < DIES_FFI_OFF || ffi > DIES_FFI_ABSORPTION) return fail(DIES_EINVAL, "unknown forced-interaction mode %d", ffi);
  m->p.k_bg = k_bg;
  m->p.ffi = ffi;
  return DIES_OK;
}

static int set_weighting_ex(Problem &p, const dies_weighting *w) {
  if (!w) return fail(DIES_EINVAL, "weighting is NULL");
  if (!(w->k_bg > 0.0 && w->k_bg <= 1.0)) return fail(DIES_EINVAL, "k_bg must lie in (0, 1]");
  if (w->forced_first_interaction < DIES_FFI_OFF || w->forced_first_interaction > DIES_FFI_ABSORPTION)
    return fail(DIES_EINVAL, "unknown forced-interaction mode %d", w->forced_first_interaction);
  if (!(std::fabs(w->g_E) < 1.0)) return fail(DIES_EINVAL, "g_E must lie in (-1, 1)");
  if (!(std::fabs(w->g_S) < 1.0)) return fail(DIES_EINVAL, "g_S must lie in (-1, 1)");
  if (!(w->k_A > 0.0 && std::isfinite(w->k_A)) || !(w->k_S > 0.0 && std::isfinite(w->k_S)))
    return fail(DIES_EINVAL, "k_A and k_S must be finite and > 0");
  if (w->k_A_density && !(w->k_A_low_density > 0.0 && std::isfinite(w->k_A_low_density) &&
                          w->k_A_high_density > 0.0 && std::isfinite(w->k_A_high_density)))
    return fail(DIES_EINVAL, "k_A_low_density and k_A_high_density must be finite and > 0");
  p.k_bg = w->k_bg;
  p.ffi = w->forced_first_interaction;
  p.g_E = w->g_E;
  p.scat_w = w->scatter_weighting ? 1 : 0;
  p.g_S = w->g_S;
  p.k_A = w->k_A;
  p.k_S = w->k_S;
  p.kA_rho = w->k_A_density ? 1 : 0;
  p.kA_lo = w->k_A_low_density;
  p.kA_hi = w->k_A_high_density;
  p.remit_random = w->reemit_uniform_in_cell ? 1 : 0;
  p.tables_valid = false;
  return DIES_OK;
}

int dies_set_weighting_ex(dies_model *m, const dies_weighting *w) {
  if (!m) return fail(DIES_EINVAL, "model is NULL");
  return set_weighting_ex(m->p, w);
}

static int set_precision(Problem &p, int mode, int n_batches, double fp64_radius) {
  if (mode != DIES_PREC_MIXED && mode != DIES_PREC_FP32 && mode != DIES_PREC_FP64)
    return fail(DIES_EINVAL, "unknown precision mode %d", mode);
  if (n_batches < 1 || n_batches > 1000000) return fail(DIES_EINVAL, "n_batches must be in [1, 1e6]");
  if (!(fp64_radius >= 0.0 && fp64_radius <= 1.0)) return fail(DIES_EINVAL, "fp64_radius must lie in [0, 1]");
  p.prec = mode;
  p.n_batches = n_batches;
  p.fp64_radius = fp64_radius;
  p.tables_valid = false;
  return DIES_OK;
}

int dies_set_precision(dies_model *m, int mode, int n_batches, double fp64_radius) {
  if (!m) return fail(DIES_EINVAL, "model is NULL");
  return set_precision(m->p, mode, n_batches, fp64_radius);
}

int dies_batch_set_precision(dies_batch *b, int mode, int n_batches, double fp64_radius) {
  if (!b) return fail(DIES_EINVAL, "batch is NULL");
  return set_precision(b->p, mode, n_batches, fp64_radius);
}

int dies_set_tgrid(dies_model *m, double T_min, double T_max, int n_nodes) {
  if (!m) return fail(DIES_EINVAL, "model is NULL");
  if (!(std::isfinite(T_min) && std::isfinite(T_max) && T_min > 0.0 && T_max > T_min))
    return fail(DIES_EINVAL, "need 0 < T_min < T_max");
  if (n_nodes < 16 || n_nodes > DIES_MAX_TNODES) return fail(DIES_EINVAL, "n_nodes must be in [16, %d]", DIES_MAX_TNODES);
  m->p.T_min = T_min;
  m->p.T_max = T_max;
  m->p.n_tnodes = n_nodes;
  m->p.tables_valid = false;
  return DIES_OK;
}

int dies_set_stream(dies_model *m, void *s) {
  if (!m) return fail(DIES_EINVAL, "model is NULL");
  m->p.stream = (cudaStream_t)s;
  return DIES_OK;
}

static int check_launch(int block, int bps, int rare_batch, int inner, int agg) {
  if (block < 64 || block > 256 || block % 32) return fail(DIES_EINVAL, "block_size must be a multiple of 32 in [64, 256]");
  if (bps < 0) return fail(DIES_EINVAL, "blocks_per_sm must be >= 0");
  if (rare_batch < 1 || rare_batch > 32) return fail(DIES_EINVAL, "rare_batch must be in [1, 32]");
  if (inner < 1 || inner > 64) return fail(DIES_EINVAL, "inner_moves must be in [1, 64]");
  if (agg != 0 && agg != 1) return fail(DIES_EINVAL, "aggregate_atomics must be 0 or 1");
  return DIES_OK;
}

static int set_launch(Problem &p, int block, int bps, int rare_batch, int inner, int agg) {
  int rc = check_launch(block, bps, rare_batch, inner, agg);
  if (rc) return rc;
  p.block = block;
  p.blocks_per_sm = bps;
  p.rare_batch = rare_batch;
  p.inner = inner;
  p.agg = agg;
  return DIES_OK;
}

int dies_set_launch(dies_model *m, int block_size, int blocks_per_sm, int rare_batch, int inner_moves,
                    int aggregate_atomics) {
  if (!m) return fail(DIES_EINVAL, "model is NULL");
  return set_launch(m->p, block_size, blocks_per_sm, rare_batch, inner_moves, aggregate_atomics);
}

static int set_launch_ex(Problem &p, const dies_launch *l) {
  if (!l) return fail(DIES_EINVAL, "launch is NULL");
  if (l->refill_divisor < 0 || l->refill_divisor > 4096)
    return fail(DIES_EINVAL, "refill_divisor must be in [0, 4096]");
  if (l->packages_per_thread < 0 || l->packages_per_thread > 2)
    return fail(DIES_EINVAL, "packages_per_thread must be 0, 1 or 2");
  if (l->reemit_table != DIES_TABLE_ALIAS && l->reemit_table != DIES_TABLE_CDF)
    return fail(DIES_EINVAL, "reemit_table must be DIES_TABLE_ALIAS or DIES_TABLE_CDF");
  if (l->stage_geometry != 0 && l->stage_geometry != 1) return fail(DIES_EINVAL, "stage_geometry must be 0 or 1");
  int rc = set_launch(p, l->block_size, l->blocks_per_sm, l->rare_batch, l->inner_moves, l->aggregate_atomics);
  if (rc) return rc;
  p.refill_div = l->refill_divisor;
  p.pkgs_per_thread = l->packages_per_thread == 2 ? 2 : 1;
  p.remit_table = l->reemit_table;
  p.stage_geo = l->stage_geometry;
  return DIES_OK;
}

int dies_set_launch_ex(dies_model *m, const dies_launch *launch) {
  if (!m) return fail(DIES_EINVAL, "model is NULL");
  return set_launch_ex(m->p, launch);
}

int dies_set_package_range(dies_model *m, uint64_t first, uint64_t count, int resume) {
  if (!m) return fail(DIES_EINVAL, "model is NULL");
  if (count == 0) return fail(DIES_EINVAL, "count must be >= 1");
  if (resume != 0 && resume != 1) return fail(DIES_EINVAL, "resume must be 0 or 1");
  m->p.range_set = true;
  m->p.range_first = first;
  m->p.range_count = count;
  m->p.range_resume = resume != 0;
  return DIES_OK;
}

int dies_set_time_budget(dies_model *m, double seconds) {
  if (!m) return fail(DIES_EINVAL, "model is NULL");
  if (!(seconds > 0.0 && seconds < 1e6)) return fail(DIES_EINVAL, "time budget must lie in (0, 1e6) s");
  m->p.time_budget_s = seconds;
  return DIES_OK;
}

int dies_set_graph(dies_model *m, int enable) {
  if (!m) return fail(DIES_EINVAL, "model is NULL");
  if (enable != 0 && enable != 1) return fail(DIES_EINVAL, "enable must be 0 or 1");
  m->p.use_graph = enable != 0;
  return DIES_OK;
}

int dies_workspace_bytes(const dies_model *m, size_t *bytes) {
  if (!m || !bytes) return fail(DIES_EINVAL, "NULL argument");
  *bytes = m->p.layout().total;
  return DIES_OK;
}

int dies_set_workspace(dies_model *m, void *ptr, size_t bytes) {
  if (!m || !ptr) return fail(DIES_EINVAL, "NULL argument");
  if (((uintptr_t)ptr & 255u) != 0) return fail(DIES_EINVAL, "workspace must be 256-byte aligned");
  const size_t need = m->p.layout().total;
  if (bytes < need) return fail(DIES_ENOMEM, "workspace of %zu bytes is smaller than the %zu needed", bytes, need);
  Problem &p = m->p;
  if (p.ws_owned && p.ws) cudaFree(p.ws);
  p.ws = (unsigned char *)ptr;
  p.ws_bytes = bytes;
  p.ws_owned = false;
  p.tables_valid = false;
  p.has_result = false;
  return DIES_OK;
}

int dies_run_async(dies_model *m, uint64_t n, uint64_t seed) {
  if (!m) return fail(DIES_EINVAL, "model is NULL");
  return m->p.enqueue_run(n, seed);
}

int dies_run(dies_model *m, uint64_t n, uint64_t seed) {
  int rc = dies_run_async(m, n, seed);
  if (rc) return rc;
  return m->p.collect();
}

int dies_get_temperatures(dies_model *m, double *T, int n) {
  if (!m) return fail(DIES_EINVAL, "model is NULL");
  return m->p.get_cells(m->p.lay.T, T, n);
}

int dies_get_absorbed(dies_model *m, double *E, int n) {
  if (!m) return fail(DIES_EINVAL, "model is NULL");
  Problem &p = m->p;
  if (p.e_in_fp32_counters && p.has_result) {
    // FP32 form: the absorbed energy is the sum of the two FP32 counters
    if (!E) return fail(DIES_EINVAL, "output pointer is NULL");
    if (n != p.n_cells) return fail(DIES_EINVAL, "expected %d shells, got %d", p.n_cells, n);
    int rc = p.collect();
    if (rc && rc != DIES_ETIMEOUT && rc != DIES_ERANGE) return rc;
    std::vector<float> a(n), b(n);
    DIES_CUDA(cudaMemcpy(a.data(), p.ws + p.lay.Eprev, (size_t)n * 4, cudaMemcpyDeviceToHost));
    // the current-batch counter of cell i sits at i * kCStride
    DIES_CUDA(cudaMemcpy2D(b.data(), 4, p.ws + p.lay.Ecur, dies::kAccSpreadBytes, 4, (size_t)n, cudaMemcpyDeviceToHost));
    for (int i = 0; i < n; ++i) E[i] = (double)a[i] + (double)b[i];
    return rc;
  }
  return p.get_cells(p.lay.E, E, n);
}

int dies_get_escaping_sed(dies_model *m, double *L, int n) {
  if (!m) return fail(DIES_EINVAL, "model is NULL");
  return m->p.get_sed(L, n);
}

int dies_get_stats(dies_model *m, dies_stats *out) {
  if (!m || !out) return fail(DIES_EINVAL, "NULL argument");
  int rc = m->p.collect();
  if (rc && rc != DIES_ETIMEOUT && rc != DIES_ERANGE) return rc;
  *out = m->p.stats;
  return rc;
}

int dies_run_frozen(dies_model *m, const double *T_frozen, uint64_t n, uint64_t seed, int flags,
                    uint32_t *n_events_out, uint64_t *path_hash_out) {
  if (!m) return fail(DIES_EINVAL, "model is NULL");
  return m->p.frozen(T_frozen, n, seed, flags, n_events_out, path_hash_out);
}

void dies_destroy_model(dies_model *m) { delete m; }

}  // extern "C"

// ------------------------------------------------ frozen pass, no allocation
// Scratch of dies_run_frozen_static: the per-shell re-emission CDF rows, then
// the work counter, event counters, energy sums, status word and escaping SED.  Host code
// must not use the symbol as an address; it looks the device address up once
// per device below.
namespace {
constexpr size_t kStaticCdfBytes = (size_t)DIES_STATIC_MAX_SHELLS * dies::kMaxFreq * 8;
constexpr size_t kStaticCounters = kStaticCdfBytes;         // 16 x u64
constexpr size_t kStaticEnergies = kStaticCdfBytes + 128;   // 8 x double
constexpr size_t kStaticQueue = kStaticCdfBytes + 192;      // 2 x u64
constexpr size_t kStaticStatus = kStaticCdfBytes + 208;     // u32
constexpr size_t kStaticDiag = kStaticCdfBytes + 256;       // 16 x u32
constexpr size_t kStaticSed = kStaticCdfBytes + 320;        // 64 x double: the escaping SED
constexpr size_t kStaticZeroBytes = 320 + 64 * 8;           // counters .. SED
static_assert(kStaticCdfBytes + kStaticZeroBytes <= DIES_STATIC_SCRATCH_BYTES, "static scratch too small");
}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[DIES_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
// per device: the scratch array's device address once looked up (null before);
// threads racing on the first lookup store the same value
std::atomic<unsigned char *> g_static_addr[kMaxDevices];

// Device address of the scratch array on the current device (looked up on the
// first call per device).
int static_scratch(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(DIES_ECUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(DIES_ECUDA, "device index %d out of range", dev);
  unsigned char *a = g_static_addr[dev].load(std::memory_order_acquire);
  if (a == nullptr) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(DIES_ECUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
    a = static_cast<unsigned char *>(p);
    g_static_addr[dev].store(a, std::memory_order_release);
  }
  *out = a;
  return DIES_OK;
}
}  // namespace

extern "C" {

int dies_run_frozen_static(dies_model *m, const double *T_frozen_dev, uint64_t n, uint64_t seed, int flags,
                           double *E_abs_dev, double *sed_dev, uint32_t *n_events_dev, uint64_t *path_hash_dev) {
  using namespace dies;
  if (!m) return fail(DIES_EINVAL, "model is NULL");
  Problem &p = m->p;
  if (!T_frozen_dev || !E_abs_dev || !sed_dev) return fail(DIES_EINVAL, "T_frozen_dev, E_abs_dev and sed_dev are required");
  if (n == 0) return fail(DIES_EINVAL, "n_packages must be >= 1");
  if (flags != DIES_FROZEN_REEMIT && flags != DIES_FROZEN_ABSORB_TERMINAL)
    return fail(DIES_EINVAL, "unknown frozen flags %d", flags);
  if (p.n_cells > DIES_STATIC_MAX_SHELLS)
    return fail(DIES_EINVAL, "%d shells exceed the static scratch capacity of %d shells", p.n_cells,
                DIES_STATIC_MAX_SHELLS);
  if (!p.ws || !p.tables_valid || p.sm_count == 0)
    return fail(DIES_ESTATE, "handle has no device tables yet: run dies_run or dies_run_async on it once first");
  unsigned char *scr = nullptr;
  int rc = static_scratch(&scr);
  if (rc) return rc;
  const unsigned long long launches0 = dies::g_launches.load();
  DIES_CUDA(cudaMemsetAsync(scr + kStaticCounters, 0, kStaticZeroBytes, p.stream));
  DIES_CUDA(cudaMemsetAsync(E_abs_dev, 0, (size_t)p.n_cells * 8, p.stream));
  double *cdf = reinterpret_cast<double *>(scr);
  DIES_CUDA(launch_frozen_cdf(p.stream, p.n_cells, p.F, p.at<double>(p.lay.freq), p.at<double>(p.lay.kabs),
                              p.at<double>(p.lay.dnu), T_frozen_dev, cdf));
  int occ = 0;
  DIES_CUDA(transport_occupancy(PREC_FP64, MODE_FROZEN, p.block, next_pow2(p.n_tnodes), false, false, false, false,
                                false, false, 0, &occ));
  if (occ < 1) return fail(DIES_ECUDA, "transport kernel cannot be resident with block size %d", p.block);
  const int bps = (p.blocks_per_sm > 0 && p.blocks_per_sm < occ) ? p.blocks_per_sm : occ;
  const int mode = (flags == DIES_FROZEN_ABSORB_TERMINAL) ? MODE_FROZEN_TERMINAL : MODE_FROZEN;
  TransportParams P = p.params(mode, n, seed);
  P.E = E_abs_dev;
  P.sed = reinterpret_cast<double *>(scr + kStaticSed);  // copied to sed_dev below
  P.cell_cdf = cdf;
  P.rec_events = n_events_dev;
  P.rec_hash = reinterpret_cast<unsigned long long *>(path_hash_dev);
  P.counters = reinterpret_cast<unsigned long long *>(scr + kStaticCounters);
  P.energies = reinterpret_cast<double *>(scr + kStaticEnergies);
  P.queue = reinterpret_cast<unsigned long long *>(scr + kStaticQueue);
  P.status = reinterpret_cast<uint32_t *>(scr + kStaticStatus);
  P.diag = reinterpret_cast<uint32_t *>(scr + kStaticDiag);
  const bool record = n_events_dev || path_hash_dev;
  DIES_CUDA(launch_transport(PREC_FP64, mode, record, P, p.sm_count * bps, p.block, p.stream));
  DIES_CUDA(cudaMemcpyAsync(sed_dev, scr + kStaticSed, (size_t)p.F * 8, cudaMemcpyDeviceToDevice, p.stream));
  // dies_get_stats on this handle reads the pass's status and counters from the scratch
  p.launches_at_start = launches0;
  p.static_counters = scr + kStaticCounters;
  p.static_energies = scr + kStaticEnergies;
  p.static_status = scr + kStaticStatus;
  p.static_diag = scr + kStaticDiag;
  p.static_sed = scr + kStaticSed;
  p.has_result = true;
  p.stats_pending = true;
  p.static_pending = true;
  return DIES_OK;
}

// ------------------------------------------------------------------ batch
int dies_create_batch(int n_models, const int *off, const double *radii, const double *rho, const int *kind,
                      double length_unit_cm, dies_batch **out) {
  if (!out) return fail(DIES_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_models < 1 || !off || !radii || !rho || !kind) return fail(DIES_EINVAL, "invalid batch arguments");
  if (off[0] != 0) return fail(DIES_EINVAL, "shell_offsets[0] must be 0");
  for (int i = 0; i < n_models; ++i) {
    const int n = off[i + 1] - off[i];
    int rc = check_geometry(radii + off[i] + i, n + 1, rho + off[i], n, length_unit_cm);
    if (rc) return fail(rc, "model %d: %s", i, dies_last_error());
    if (kind[i] < 1 || kind[i] > 3) return fail(DIES_EINVAL, "source_kind[%d] must be 1, 2 or 3", i);
  }
  dies_batch *b = new (std::nothrow) dies_batch();
  if (!b) return fail(DIES_ENOMEM, "host allocation failed");
  Problem &p = b->p;
  p.n_models = n_models;
  p.n_cells = off[n_models];
  p.radii.assign(radii, radii + off[n_models] + n_models);
  p.rho.assign(rho, rho + off[n_models]);
  p.kind.assign(kind, kind + n_models);
  p.length_unit_cm = length_unit_cm;
  p.desc.resize(n_models);
  for (int i = 0; i < n_models; ++i) {
    p.desc[i] = dies::ModelDesc{};
    p.desc[i].cell_off = off[i];
    p.desc[i].bnd_off = off[i] + i;
    p.desc[i].n_cells = off[i + 1] - off[i];
  }
  *out = b;
  return DIES_OK;
}

int dies_batch_set_dust(dies_batch *b, const double *freq_hz, int n_freq, const double *ka, const double *ks,
                        const double *g) {
  if (!b) return fail(DIES_EINVAL, "batch is NULL");
  return b->p.set_dust(freq_hz, n_freq, ka, ks, g);
}

int dies_batch_set_sources(dies_batch *b, const double *J_ext, double L_point, const double *spec) {
  if (!b) return fail(DIES_EINVAL, "batch is NULL");
  return b->p.set_sources(J_ext, L_point, spec);
}

int dies_batch_set_stream(dies_batch *b, void *s) {
  if (!b) return fail(DIES_EINVAL, "batch is NULL");
  b->p.stream = (cudaStream_t)s;
  return DIES_OK;
}

int dies_batch_set_launch(dies_batch *b, int block_size, int blocks_per_sm, int rare_batch, int inner_moves,
                          int aggregate_atomics) {
  if (!b) return fail(DIES_EINVAL, "batch is NULL");
  return set_launch(b->p, block_size, blocks_per_sm, rare_batch, inner_moves, aggregate_atomics);
}

int dies_batch_set_launch_ex(dies_batch *b, const dies_launch *launch) {
  if (!b) return fail(DIES_EINVAL, "batch is NULL");
  return set_launch_ex(b->p, launch);
}

int dies_batch_set_weighting(dies_batch *b, const dies_weighting *w) {
  if (!b) return fail(DIES_EINVAL, "batch is NULL");
  return set_weighting_ex(b->p, w);
}

int dies_batch_set_graph(dies_batch *b, int enable) {
  if (!b) return fail(DIES_EINVAL, "batch is NULL");
  if (enable != 0 && enable != 1) return fail(DIES_EINVAL, "enable must be 0 or 1");
  b->p.use_graph = enable != 0;
  return DIES_OK;
}

int dies_run_batch_async(dies_batch *b, uint64_t n, uint64_t seed) {
  if (!b) return fail(DIES_EINVAL, "batch is NULL");
  return b->p.enqueue_run(n, seed);
}

int dies_run_batch(dies_batch *b, uint64_t n, uint64_t seed) {
  int rc = dies_run_batch_async(b, n, seed);
  if (rc) return rc;
  return b->p.collect();
}

int dies_batch_get_temperatures(dies_batch *b, double *T, int n) {
  if (!b) return fail(DIES_EINVAL, "batch is NULL");
  return b->p.get_cells(b->p.lay.T, T, n);
}

int dies_batch_get_escaping_sed(dies_batch *b, double *L, int n) {
  if (!b) return fail(DIES_EINVAL, "batch is NULL");
  return b->p.get_sed(L, n);
}

int dies_batch_get_stats(dies_batch *b, dies_stats *out) {
  if (!b || !out) return fail(DIES_EINVAL, "NULL argument");
  int rc = b->p.collect();
  if (rc && rc != DIES_ETIMEOUT && rc != DIES_ERANGE) return rc;
  *out = b->p.stats;
  return rc;
}

void dies_destroy_batch(dies_batch *b) { delete b; }

const char *dies_last_error(void) { return dies::t_error.c_str(); }

uint64_t dies_launch_count(void) { return dies::g_launches.load(); }

#ifdef DIES_CHECK
const char *dies_version(void) { return "dies-gb300 0.2 (sm_103a, device bounds checks)"; }
#else
const char *dies_version(void) { return "dies-gb300 0.2 (sm_103a)"; }
#endif

}  // extern "C"
