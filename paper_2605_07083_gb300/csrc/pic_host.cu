// pic_host.cu -- host side of the C ABI declared in include/pic.h.
//
// Owns the device state of a handle, derives the per-diode constants in FP64
// (Sec. 2.1 grid and Poisson scaling, Sec. 2.2 emission and null-collision
// constants), enqueues the per-step kernels (as CUDA graphs when possible) and
// turns the device tallies into the Sec. 2.3 / Eq. 1-8 diagnostics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/pic.h"
#include "pic_internal.cuh"

namespace pic {
__global__ void k_push(DevState st);
__global__ void k_push32(DevState st);
__global__ void k_deposit(DevState st);
__global__ void k_mid(DevState st);
__global__ void k_post(DevState st);
__global__ void k_field(DevState st);
__global__ void k_profile(DevState st);
__global__ void k_phi(DevState st);
__global__ void k_fill_ids(uint32_t* id, long long n, uint32_t first);
__global__ void k_count_outside(const float* z, long long n, float Lf, int* bad);
void sort_launch(const DevState& st, int max_chunks, int max_nz, cudaStream_t s);
size_t sort_hist_ints(const int32_t* seg_cap, const int* seg_nz, int n_seg, int64_t* hoff);
int sort_max_chunks(const int32_t* seg_cap, int n_seg);
cudaError_t sort_prepare(int smem_bytes);
}  // namespace pic

using namespace pic;

namespace {

const double kQe = 1.602176634e-19;
const double kMe = 9.1093837015e-31;
const double kEps0 = 8.8541878128e-12;
const double kKb = 1.380649e-23;
const double kEionHe = 24.59;   // first ionisation energy of He (Sec. 2.4)

struct Alloc {
  void* p;
  size_t bytes;
};

}  // namespace

struct pic_handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  pic_allocator alloc{};
  bool has_alloc = false;
  int n_inst = 0, n_seg = 0;
  std::vector<pic_config> cfg;
  std::vector<InstConst> ic;
  std::vector<int64_t> seg_off;
  std::vector<int32_t> seg_cap;
  int64_t total_cap = 0;
  int total_nodes = 0, max_nodes = 0;
  int sm_count = 0;
  int push_threads = 256, blocks_per_sm = 0, G = 0;   // 0 blocks/SM: occupancy limit
  int sort_period = 0, graph_steps = 64;
  bool threads_set = false;     // push_threads chosen by the caller (pic_tune)
  int push_chunk = 64;          // quads per warp chunk of the push (64 or 32)
  bool chunk_set = false;       // push_chunk chosen by the caller (pic_tune)
  DevState st{};
  std::vector<Alloc> allocs;
  bool dirty = true;
  int sticky = PIC_OK;
  int64_t host_step = 0;        // mirror of the device step counter
  int64_t last_sort_step = 0;
  // step loops by length, longest first (plan_graphs), captured when first
  // needed, so that any step count runs as graphs
  std::vector<std::pair<int, cudaGraphExec_t>> graphs;
  size_t push_smem = 0, post_smem = 0, field_smem = 0, mid_smem = 0;
  size_t dcount_ints = 0;
  int bstart_len = 0;
  int* inject_flag = nullptr;   // device word: an injected z outside [0, L)
  int bw_len = 0;
  int mcc_blocks = 0;
  bool sort_ready = false;
  int sort_chunks = 1;
  int prof_gx = 1;              // k_profile blocks per segment
  size_t prof_smem = 0;
  char last_error[256] = {0};
};

namespace {

int cuda_fail_at(pic_handle* h, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return PIC_OK;
  if (h && h->sticky == PIC_OK) {
    h->sticky = PIC_ECUDA;
    std::snprintf(h->last_error, sizeof(h->last_error), "%s: %s", where, cudaGetErrorString(e));
  }
  return e == cudaErrorMemoryAllocation ? PIC_ENOMEM : PIC_ECUDA;
}
#define cuda_fail(h, e) cuda_fail_at((h), (e), __func__)

void* dev_alloc(pic_handle* h, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  if (h->has_alloc) {
    p = h->alloc.alloc(bytes, (void*)h->stream, h->alloc.ctx);
  } else if (cudaMallocAsync(&p, bytes, h->stream) != cudaSuccess) {
    p = nullptr;
  }
  if (p) h->allocs.push_back({p, bytes});
  return p;
}

void free_all(pic_handle* h) {
  for (auto& a : h->allocs) {
    if (h->has_alloc) h->alloc.free(a.p, a.bytes, (void*)h->stream, h->alloc.ctx);
    else cudaFreeAsync(a.p, h->stream);
  }
  h->allocs.clear();
}

bool cfg_valid(const pic_config& c) {
  if (c.size != sizeof(pic_config)) return false;
  if (c.n_cells < 1 || c.n_cells > kMaxNz) return false;
  if (!(c.gap_m > 0) || !(c.dt_s > 0) || !(c.weight > 0)) return false;
  if (!(c.m_ion > 0) || !(c.m_gas > 0)) return false;
  if (!(c.gamma_emit >= 0) || !(c.T_wall_K >= 0) || !(c.n_gas >= 0)) return false;
  if (!(c.T_gas_e_K >= 0) || !(c.T_gas_i_K >= 0) || !(c.T_e0_eV >= 0) || !(c.T_i0_eV >= 0))
    return false;
  if (!(c.sigma_el_e >= 0) || !(c.sigma_cx_i >= 0) || !(c.sigma_el_i >= 0)) return false;
  if (!(c.sigma_exc0 >= 0) || !(c.lotz_a >= 0)) return false;
  if (c.n_gas > 0 && (!(c.E_cap_e_eV > 0) || !(c.E_cap_i_eV > 0))) return false;
  for (int s = 0; s < 3; ++s)
    if (c.capacity[s] < 0 || c.capacity[s] > (1LL << 30)) return false;
  const double x = c.gamma_emit * c.dt_s / c.weight;
  if (!(x < 1e8)) return false;
  return true;
}

// Per-instance constants, FP64 on the host.
InstConst derive(const pic_config& c) {
  InstConst k;
  std::memset(&k, 0, sizeof(k));
  k.Nz = c.n_cells;
  const double L = c.gap_m, dz = L / c.n_cells;
  k.inv_dz_f = (float)((double)c.n_cells / L);
  k.L_f = (float)L;
  k.dt_f = (float)c.dt_s;
  const double m[3] = {kMe, kMe, c.m_ion};
  const double q[3] = {-kQe, -kQe, kQe};
  for (int s = 0; s < 3; ++s) k.qmdt[s] = (float)(q[s] / m[s] * c.dt_s);
  k.dz = dz;
  k.inv_dz = 1.0 / dz;
  k.inv_nz = 1.0 / c.n_cells;
  k.V = c.bias_V;
  // phi per fixed-point charge unit: dz^2 * (e w / (2^24 dz)) / eps0
  k.kappa = dz * kQe * c.weight / (16777216.0 * kEps0);
  // null-collision frequency bound: n * (max over E <= E_cap of sum sigma) * g(E_cap)
  const double M = c.m_gas;
  double smax_e = c.sigma_el_e;
  if (c.sigma_exc0 > 0 && c.E_cap_e_eV > c.E_exc_eV)
    smax_e += c.sigma_exc0 * (1.0 - c.E_exc_eV / c.E_cap_e_eV);
  if (c.lotz_a > 0 && c.E_cap_e_eV > c.E_iz_eV) {
    const double P = c.E_iz_eV, e1 = std::exp(1.0), peak = P * e1;
    if (c.E_cap_e_eV >= peak) smax_e += c.lotz_a * c.lotz_q / (e1 * P * P);
    else smax_e += c.lotz_a * c.lotz_q * std::log(c.E_cap_e_eV / P) / (c.E_cap_e_eV * P);
  }
  const double smax_i = c.sigma_cx_i + c.sigma_el_i;
  for (int s = 0; s < 3; ++s) {
    const double mu = m[s] * M / (m[s] + M);
    const double Ecap = s < 2 ? c.E_cap_e_eV : c.E_cap_i_eV;
    const double gmax = std::sqrt(2.0 * Ecap * kQe / mu);
    const double numax = c.n_gas * (s < 2 ? smax_e : smax_i) * gmax;
    const double P = -std::expm1(-numax * c.dt_s);
    k.t_cand[s] = (c.n_gas <= 0 || numax <= 0) ? 0u
                  : (P >= 1.0 ? 0xFFFFFFFFu : (uint32_t)(P * 4294967296.0));
    k.nu_max[s] = (float)numax;
    const double Tn = s < 2 ? c.T_gas_e_K : c.T_gas_i_K;
    k.sig_n[s] = (float)std::sqrt(kKb * Tn / M);
    k.fm[s] = (float)(m[s] / (m[s] + M));
    k.fM[s] = (float)(M / (m[s] + M));
    k.half_mu_over_e[s] = (float)(0.5 * mu / kQe);
    k.two_e_over_mu[s] = (float)(2.0 * kQe / mu);
    k.m_d[s] = m[s];
  }
  k.two_e_over_me = (float)(2.0 * kQe / kMe);
  k.n_gas = (float)c.n_gas;
  k.sigma_el_e = (float)c.sigma_el_e;
  k.sigma_cx_i = (float)c.sigma_cx_i;
  k.sigma_el_i = (float)c.sigma_el_i;
  k.E_exc = (float)c.E_exc_eV;
  k.sigma_exc0 = (float)c.sigma_exc0;
  k.E_iz = (float)c.E_iz_eV;
  k.lotz_aq = (float)(c.lotz_a * c.lotz_q);
  const uint32_t slo = (uint32_t)c.seed, shi = (uint32_t)(c.seed >> 32);
  for (uint32_t s = 0; s < 4; ++s) k.key0[s] = slo ^ (uint32_t)(s * 0x9E3779B9u);
  k.key1 = shi;
  // candidate word: Philox2x32-10 under seed_lo ^ species*0x9E3779B9 ^ seed_hi
  for (uint32_t s = 0; s < 3; ++s) k.ckey[s] = slo ^ (uint32_t)(s * 0x9E3779B9u) ^ shi;
  // thermionic emission: N = floor(x) + [u < frac(x)], x = Gamma dt / w (Sec. 2.2)
  const double x = (c.gamma_emit * c.dt_s) / c.weight;
  const double fl = std::floor(x);
  k.emit_floor = (int64_t)fl;
  k.t_frac = (uint32_t)((x - fl) * 4294967296.0);
  k.sig_w = (float)std::sqrt(kKb * c.T_wall_K / kMe);
  k.sig_e0 = (float)std::sqrt(c.T_e0_eV * kQe / kMe);
  k.sig_i0 = (float)std::sqrt(c.T_i0_eV * kQe / c.m_ion);
  k.replenish = c.replenish ? 1 : 0;
  k.weight = c.weight;
  k.window_start = c.window_start;
  return k;
}

int64_t default_capacity(const pic_config& c, int s) {
  (void)c;
  (void)s;
  return 1 << 20;
}

int check_flags(pic_handle* h) {
  std::vector<InstDyn> dyn(h->n_inst);
  cudaError_t e = cudaMemcpyAsync(dyn.data(), h->st.dyn, sizeof(InstDyn) * h->n_inst,
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  int bits = 0;
  for (auto& d : dyn) bits |= d.err;
  if (h->sticky == PIC_OK) {
    if (bits & ERR_CAPACITY) h->sticky = PIC_ECAPACITY;
    else if (bits & ERR_TIMEOUT) h->sticky = PIC_ETIMEOUT;
    else if (bits & ERR_ENERGYCAP) h->sticky = PIC_EENERGYCAP;
  }
  return h->sticky;
}

void drop_graph(pic_handle* h) {
  for (auto& g : h->graphs)
    if (g.second) cudaGraphExecDestroy(g.second);
  h->graphs.clear();
}

// dynamic shared memory a kernel may request: the opt-in maximum less its
// static shared memory
cudaError_t set_dynamic_smem_limit(const void* f, int optin) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, f);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)a.sharedSizeBytes);
}

// The dynamic shared-memory limit is a process-wide attribute of each kernel:
// raise it once per device to the opt-in maximum, so that handles of
// different grid sizes never lower it under one another's launches.
cudaError_t raise_smem_limits(int device) {
  static bool done[64] = {false};
  if (device >= 0 && device < 64 && done[device]) return cudaSuccess;
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e != cudaSuccess) return e;
  const void* fns[] = {(const void*)k_push, (const void*)k_push32,
                       (const void*)k_deposit, (const void*)k_field,
                       (const void*)k_post, (const void*)k_profile, (const void*)k_phi,
                       (const void*)k_mid};
  for (const void* f : fns) {
    e = set_dynamic_smem_limit(f, optin);

    if (e != cudaSuccess) return e;
  }
  e = sort_prepare(optin);
  if (e == cudaSuccess && device >= 0 && device < 64) done[device] = true;
  return e;
}

size_t push_smem_bytes(const pic_handle* h, int threads, int chunk) {
  // Es2 + histogram (20 B per node), segment prefix and offsets, staging
  const size_t fixed = (size_t)h->max_nodes * 20 + 8 + (size_t)(2 * h->n_seg + 1) * 8;
  return ((fixed + 127) & ~(size_t)127) +
         (size_t)(threads / 32) * 2 * ((size_t)stage_bytes(chunk) + 8);
}

using PushKernel = void (*)(DevState);
PushKernel push_kernel(int chunk) { return chunk == 32 ? k_push32 : k_push; }

// resident warps per SM of a push shape (0 if it does not fit)
int push_warps(const pic_handle* h, int threads, int chunk) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, push_kernel(chunk), threads,
                                                    push_smem_bytes(h, threads, chunk)) !=
      cudaSuccess)
    return 0;
  return occ * threads / 32;
}

// Default push shape: the push is issue-bound, and on this part about 24
// resident warps per SM hide its latencies best (more contend for issue
// slots, fewer leave dependency waits exposed).  The shared-memory footprint
// grows with the cell count and the chunk, so pick the block size and chunk
// that get closest to 24 warps from below, preferring 64-quad chunks, then
// 384 threads (two blocks per SM), on ties.  A caller's choice of either is
// kept.
void default_push_shape(pic_handle* h) {
  int best_t = h->threads_set ? h->push_threads : 384;
  int best_c = h->chunk_set ? h->push_chunk : 64;
  int best_w = -1;
  for (int c : {64, 32}) {
    if (h->chunk_set && c != h->push_chunk) continue;
    for (int t : {384, 256, 128, 160, 192, 224, 288, 320, 352}) {
      if (h->threads_set && t != h->push_threads) continue;
      const int w = std::min(push_warps(h, t, c), 24);
      if (w > best_w) { best_t = t; best_c = c; best_w = w; }
    }
  }
  h->push_threads = best_t;
  h->push_chunk = best_c;
}

int set_launch_shape(pic_handle* h) {
  cudaError_t e = raise_smem_limits(h->device);
  if (e != cudaSuccess) return cuda_fail(h, e);
  default_push_shape(h);
  h->push_smem = push_smem_bytes(h, h->push_threads, h->push_chunk);
  h->field_smem = (size_t)h->max_nodes * 8;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, push_kernel(h->push_chunk),
                                                    h->push_threads, h->push_smem);
  if (e != cudaSuccess) return cuda_fail(h, e);
  if (occ < 1) occ = 1;
  const int per_sm = h->blocks_per_sm > 0 ? std::min(h->blocks_per_sm, occ) : occ;
  // one wave: every block resident at once (a block flushes its histogram
  // after every kSubQuads quads, so its share has no upper bound)
  h->G = h->sm_count * per_sm;
  h->st.G = h->G;
  // k_mid spreads a diode's field and a segment's absorbed list over kp
  // blocks each when the diodes are few (their FP64 work then shares no SM)
  h->st.kp = std::max(1, std::min(kMaxParts, h->sm_count / (4 * h->n_inst)));
  h->st.W = h->push_threads / 32;
  // collision blocks of k_mid: one per SM, two where the expected candidates
  // per step (candidate probability x capacity) would give every thread of
  // one block per SM more than one collision (measured: 1.2x faster k_mid at
  // ~1 % candidates of 22M particles, 0.9x at 0.01 % of 10M)
  double cand = 0.0;
  for (int i = 0; i < h->n_inst; ++i)
    for (int s = 0; s < 3; ++s)
      cand += (double)h->ic[i].t_cand[s] * (1.0 / 4294967296.0) * (double)h->seg_cap[3 * i + s];
  h->mcc_blocks = cand > (double)h->sm_count * kPostThreads ? 2 * h->sm_count : h->sm_count;
  const size_t need = (size_t)h->n_seg * h->G;
  if (need > h->dcount_ints) {
    void* p = dev_alloc(h, need * sizeof(int32_t));
    if (!p) return PIC_ENOMEM;
    h->st.dcount = (int32_t*)p;
    h->dcount_ints = need;
  }
  // push-block weights back to their starting shares; their times unknown.
  // Blocks placed in an earlier round on an SM get more of its issue slots:
  // measured on the production diode with two blocks per SM, the first
  // round settles at 1.2x and the second at 0.8x the nominal share, so the
  // shares start there (and at +-1/3 across three or more rounds, where the
  // first block ran about twice as fast as the third)
  // layout: bwp [G + 1] long long, bw [G] int, bt [G] int, bw_n [2] int
  const size_t bw_bytes = sizeof(long long) * (size_t)(2 * h->G + 2);
  if (h->G > h->bw_len) {
    void* p = dev_alloc(h, bw_bytes);
    if (!p) return PIC_ENOMEM;
    h->st.bwp = (long long*)p;
    h->bw_len = h->G;
  }
  h->st.bw = (int*)(h->st.bwp + h->G + 1);
  h->st.bt = h->st.bw + h->G;
  h->st.bw_n = h->st.bt + h->G;
  {
    std::vector<long long> w((size_t)2 * h->G + 2, 0);
    int* wi = reinterpret_cast<int*>(w.data() + h->G + 1);
    const int rounds = std::max(1, h->G / std::max(1, h->sm_count));
    const double spread = rounds == 2 ? 0.2 : 1.0 / 3.0;
    for (int b = 0; b < h->G; ++b) {
      const int k = std::min(b / std::max(1, h->sm_count), rounds - 1);
      const double f = rounds > 1 ? (rounds - 1 - 2.0 * k) / (rounds - 1) : 0.0;
      wi[b] = (int)std::lround(kNominalWeight * (1.0 + spread * f));
      w[b + 1] = w[b] + wi[b];
    }
    // the prefix in units of 2^-32 of the total, as the weights block writes it
    const unsigned long long total = (unsigned long long)w[h->G];
    for (int b = 1; b <= h->G; ++b)
      w[b] = (long long)(((unsigned long long)w[b] << 32) / total);
    const size_t bytes = bw_bytes;
    cudaError_t e2 = cudaMemcpyAsync(h->st.bwp, w.data(), bytes, cudaMemcpyHostToDevice, h->stream);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(h->stream);
    if (e2 != cudaSuccess) return cuda_fail(h, e2);
  }
  if (h->G + 1 > h->bstart_len) {
    void* p = dev_alloc(h, sizeof(int64_t) * (size_t)(h->G + 1));
    if (!p) return PIC_ENOMEM;
    h->st.bstart = (int64_t*)p;
    h->bstart_len = h->G + 1;
  }
  // k_mid: a diode's charge and emission histogram, or a segment's piece
  // ranges and prefix; k_post: the staged absorbed list or the event keys
  h->mid_smem = std::max((size_t)h->max_nodes * 20, (size_t)(h->G + 1) * 12) + 16;
  h->post_smem = std::max((size_t)kDeadSmem * 4, (size_t)kEvCap * 8) + 16;
  // profile sampler: blocks per segment so that none bins more than
  // kHistMaxParticles particles (its 32-bit counters), else about two blocks
  // per SM in total
  int64_t max_cap = 1;
  for (int32_t c : h->seg_cap) max_cap = std::max<int64_t>(max_cap, c);
  const int64_t gmin = (max_cap + kHistMaxParticles - 1) / kHistMaxParticles;
  const int64_t gfill = std::min<int64_t>((max_cap + 8191) / 8192,
                                          std::max<int64_t>(1, 2 * h->sm_count / h->n_seg));
  h->prof_gx = (int)std::max<int64_t>(1, std::max(gmin, gfill));
  h->prof_smem = (size_t)(h->max_nodes - 1) * 12;
  drop_graph(h);
  return PIC_OK;
}

// scratch of the counting sort: a second particle set and the histograms
int sort_alloc(pic_handle* h) {
  if (h->sort_ready) return PIC_OK;
  const size_t P = (size_t)h->total_cap;
  std::vector<int> nz(h->n_seg);
  std::vector<int64_t> hoff(h->n_seg);
  for (int g = 0; g < h->n_seg; ++g) nz[g] = h->cfg[g / 3].n_cells;
  const size_t hist = sort_hist_ints(h->seg_cap.data(), nz.data(), h->n_seg, hoff.data());
  void* a = dev_alloc(h, P * 4 * 5);
  void* b = dev_alloc(h, hist * 4);
  void* c = dev_alloc(h, sizeof(int64_t) * h->n_seg);
  if (!a || !b || !c) return PIC_ENOMEM;
  h->st.z2 = (float*)a;
  h->st.vx2 = h->st.z2 + P;
  h->st.vy2 = h->st.vx2 + P;
  h->st.vz2 = h->st.vy2 + P;
  h->st.id2 = (uint32_t*)(h->st.vz2 + P);
  h->st.sort_hist = (int32_t*)b;
  h->st.sort_hoff = (const int64_t*)c;
  cudaError_t e = cudaMemcpyAsync(c, hoff.data(), sizeof(int64_t) * h->n_seg, cudaMemcpyHostToDevice,
                                  h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  h->sort_chunks = sort_max_chunks(h->seg_cap.data(), h->n_seg);
  h->sort_ready = true;
  drop_graph(h);
  return PIC_OK;
}

void launch_sort(pic_handle* h) { sort_launch(h->st, h->sort_chunks, h->max_nodes, h->stream); }

cudaError_t launch_field(pic_handle* h) {
  k_deposit<<<h->G, h->push_threads, h->push_smem, h->stream>>>(h->st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_field<<<h->n_inst, kPostThreads, h->field_smem, h->stream>>>(h->st);
  return cudaGetLastError();
}

int ensure_field(pic_handle* h) {
  if (!h->dirty) return PIC_OK;
  cudaError_t e = launch_field(h);
  if (e != cudaSuccess) return cuda_fail_at(h, e, "k_deposit/k_field launch");
  h->dirty = false;
  return PIC_OK;
}

bool sort_due(const pic_handle* h, int64_t step_after) {
  return h->sort_period > 0 && step_after % h->sort_period == 0;
}

// k_mid: kp field blocks per diode, kp list blocks per segment, one block
// for the push weights, then the collision blocks
int mid_blocks(const pic_handle* h) { return 4 * h->n_inst * h->st.kp + 1 + h->mcc_blocks; }

// the profile sampler after a step (device-side test of the sampling rule)
void launch_profile(pic_handle* h) {
  if (h->st.prof_period > 0)
    k_profile<<<dim3((unsigned)h->prof_gx, (unsigned)h->n_seg), 256, h->prof_smem, h->stream>>>(h->st);
}

// one time step; the sort, when due, follows the step
cudaError_t launch_step(pic_handle* h) {
  push_kernel(h->push_chunk)<<<h->G, h->push_threads, h->push_smem, h->stream>>>(h->st);
  k_mid<<<mid_blocks(h), kPostThreads, h->mid_smem, h->stream>>>(h->st);
  k_post<<<3 * h->n_inst, kPostThreads, h->post_smem, h->stream>>>(h->st);
  launch_profile(h);
  h->host_step += 1;
  if (sort_due(h, h->host_step)) launch_sort(h);
  return cudaGetLastError();
}

// Captures len steps.  With a periodic sort the graph is only ever launched
// on a sort-aligned step, so the sorts sit after every sort_period-th step of
// it counted from its start.
int build_graph(pic_handle* h, int len, cudaGraphExec_t* out) {
  *out = nullptr;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail_at(h, e, "cudaStreamBeginCapture");
  for (int i = 0; i < len; ++i) {
    push_kernel(h->push_chunk)<<<h->G, h->push_threads, h->push_smem, h->stream>>>(h->st);
    k_mid<<<mid_blocks(h), kPostThreads, h->mid_smem, h->stream>>>(h->st);
    k_post<<<3 * h->n_inst, kPostThreads, h->post_smem, h->stream>>>(h->st);
    launch_profile(h);
    if (sort_due(h, i + 1)) launch_sort(h);
  }
  e = cudaStreamEndCapture(h->stream, &g);
  if (e != cudaSuccess) return cuda_fail_at(h, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *out = nullptr;
    return cuda_fail_at(h, e, "cudaGraphInstantiate");
  }
  return PIC_OK;
}

// Length of the longest step graph: graph_steps, at most kMaxGraphSteps,
// rounded up to a multiple of the sort period when there is one; 0 (no
// graphs) when graphs are off or a sort period is longer than the cap.
constexpr int kMaxGraphSteps = 4096;
int graph_unit(const pic_handle* h) {
  if (h->graph_steps <= 0) return 0;
  const int64_t want = std::min(h->graph_steps, kMaxGraphSteps);
  if (h->sort_period <= 0) return (int)want;
  const int64_t sp = h->sort_period;
  const int64_t len = (want + sp - 1) / sp * sp;
  return len <= kMaxGraphSteps ? (int)len : 0;
}

// The step graphs' lengths, longest first: graph_unit, then u * 2^k for
// every u * 2^k below it, u = 1 without a sort and u = sort_period with one.
// pic_step runs any step count as graphs of these lengths, less at most
// sort_period - 1 single steps on each side when a sort is on.  Each graph
// is captured the first time a pic_step needs it.
void plan_graphs(pic_handle* h) {
  drop_graph(h);
  const int top = graph_unit(h);
  const int unit = h->sort_period > 0 ? h->sort_period : 1;
  h->graphs.push_back({top, nullptr});
  int64_t p = unit;
  while (p * 2 < top) p *= 2;
  for (; p >= unit; p /= 2)
    if (p < top) h->graphs.push_back({(int)p, nullptr});
}

void fill_diag(const pic_handle* h, int inst, const InstDyn& d, const int32_t* counts,
               pic_diag* o) {
  const pic_config& c = h->cfg[inst];
  std::memset(o, 0, sizeof(*o));
  o->step = d.step;
  o->window_steps = d.win_steps;
  const double T = (double)d.win_steps * c.dt_s;
  o->window_time = T;
  for (int s = 0; s < 3; ++s) {
    o->n_live[s] = counts[s];
    o->candidates[s] = (int64_t)d.cand[s];
    for (int w = 0; w < 2; ++w) {
      o->count[s][w] = d.count[s][w];
      o->ke[s][w] = d.ke[s][w];
    }
  }
  for (int k = 0; k < 6; ++k) o->collisions[k] = (int64_t)d.coll[k];
  o->emitted = d.emitted;
  o->replenished = d.replenished;
  o->energy_cap_exceeded = (int64_t)d.cap_exceeded;
  o->particles_pushed = d.pushed;
  o->error_flags = d.err;
  const double w = c.weight;
  o->gamma_emit = c.gamma_emit;
  o->T_c_eV = kKb * c.T_wall_K / kQe;
  if (T <= 0) return;
  // Sec. 2.3 fluxes of the emitted population
  o->gamma_emit_realized = (double)d.emitted * w / T;
  o->gamma_ref = (double)d.count[0][0] * w / T;
  o->gamma_anode = (double)d.count[0][1] * w / T;
  o->gamma_net = c.gamma_emit - o->gamma_ref;
  if (c.gamma_emit > 0) {
    o->backflow_ratio = o->gamma_ref / c.gamma_emit;
    o->net_efficiency = o->gamma_net / c.gamma_emit;
    o->collection_efficiency = o->gamma_anode / c.gamma_emit;
  }
  // Eq. 2: effective work function from Richardson-Dushman with
  // A_R = 1.20e6 / (k_B/e)^2 (A m^-2 eV^-2); Eq. 1: emitted cooling power
  const double kbe = kKb / kQe;
  const double AR = 1.20e6 / (kbe * kbe);
  const double Tc = o->T_c_eV;
  if (c.gamma_emit > 0 && Tc > 0) {
    o->W_F_eff = -Tc * std::log(kQe * c.gamma_emit / (AR * Tc * Tc));
    o->q_emit_theory = c.gamma_emit * kQe * (o->W_F_eff + 2.0 * Tc);
  }
  o->q_back_em_cath = d.ke[0][0] / T;
  o->q_back_p_cath = d.ke[1][0] / T;
  o->q_ion_cath = d.ke[2][0] / T;
  o->gamma_ion_cath = (double)d.count[2][0] * w / T;
  o->q_ion_cath_recomb = o->gamma_ion_cath * kQe * kEionHe;                 // Eq. 3
  o->q_cooling_1 = o->q_emit_theory - o->q_back_em_cath - o->q_back_p_cath - o->q_ion_cath;  // Eq. 4
  o->q_cooling_2 = o->q_cooling_1 - o->q_ion_cath_recomb;                   // Eq. 5
  o->q_out_em_anode = d.ke[0][1] / T;
  o->q_out_p_anode = d.ke[1][1] / T;
  o->q_ion_anode = d.ke[2][1] / T;
  o->q_anode_total_1 = o->q_out_em_anode + o->q_out_p_anode + o->q_ion_anode;  // Eq. 6
  o->gamma_ion_anode = (double)d.count[2][1] * w / T;
  o->q_ion_anode_recomb = o->gamma_ion_anode * kQe * kEionHe;               // Eq. 7
  o->q_anode_total_2 = o->q_anode_total_1 + o->q_ion_anode_recomb;          // Eq. 8
}


}  // namespace

extern "C" {

int pic_abi_version(void) { return PIC_ABI_VERSION; }

size_t pic_sizeof(int which) {
  switch (which) {
    case 0: return sizeof(pic_config);
    case 1: return sizeof(pic_tuning);
    case 2: return sizeof(pic_diag);
    case 3: return sizeof(pic_profile);
    case 4: return sizeof(pic_vc);
    default: return 0;
  }
}

const char* pic_strerror(int code) {
  switch (code) {
    case PIC_OK: return "ok";
    case PIC_EINVAL: return "invalid argument or configuration";
    case PIC_ENOMEM: return "device allocation failed";
    case PIC_ECUDA: return "CUDA runtime error";
    case PIC_ECAPACITY: return "particle or event capacity exceeded";
    case PIC_ETIMEOUT: return "bounded device wait timed out";
    case PIC_EENERGYCAP: return "collision energy above the null-collision bound";
    default: return "unknown error";
  }
}

int pic_create(const pic_config* cfgs, int n_instances, void* cuda_stream,
               const pic_allocator* alloc, pic_handle** out) {
  if (!out) return PIC_EINVAL;
  *out = nullptr;
  if (!cfgs || n_instances < 1 || n_instances > kMaxInstances) return PIC_EINVAL;
  for (int i = 0; i < n_instances; ++i)
    if (!cfg_valid(cfgs[i])) return PIC_EINVAL;
  if (alloc && (!alloc->alloc || !alloc->free)) return PIC_EINVAL;

  pic_handle* h = new pic_handle();
  if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return PIC_ECUDA; }
  cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
  if (h->sm_count <= 0) h->sm_count = 1;
  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return PIC_ECUDA;
    }
    h->own_stream = true;
  }
  if (alloc) { h->alloc = *alloc; h->has_alloc = true; }
  h->n_inst = n_instances;
  h->n_seg = 3 * n_instances;
  h->cfg.assign(cfgs, cfgs + n_instances);
  h->ic.resize(n_instances);
  h->seg_off.resize(h->n_seg);
  h->seg_cap.resize(h->n_seg);
  int64_t off = 0;
  int nodes = 0;
  for (int i = 0; i < n_instances; ++i) {
    h->ic[i] = derive(cfgs[i]);
    h->ic[i].node_off = nodes;
    nodes += ((cfgs[i].n_cells + 1 + 31) / 32) * 32;
    h->max_nodes = std::max(h->max_nodes, cfgs[i].n_cells + 1);
    for (int s = 0; s < 3; ++s) {
      int64_t cap = cfgs[i].capacity[s] > 0 ? cfgs[i].capacity[s] : default_capacity(cfgs[i], s);
      cap = ((cap + 31) / 32) * 32;
      h->seg_off[3 * i + s] = off;
      h->seg_cap[3 * i + s] = (int32_t)cap;
      off += cap;
    }
  }
  h->total_cap = off;
  h->total_nodes = nodes;
  if (h->total_cap > kMaxSlots) { pic_destroy(h); return PIC_EINVAL; }

  DevState& st = h->st;
  st.n_inst = h->n_inst;
  st.wait_limit = kWaitLimit;
  st.n_seg = h->n_seg;
  st.max_nodes = h->max_nodes;
  const size_t P = (size_t)h->total_cap;
  void* p[16] = {nullptr};
  p[0] = dev_alloc(h, P * 4); p[1] = dev_alloc(h, P * 4); p[2] = dev_alloc(h, P * 4);
  p[3] = dev_alloc(h, P * 4); p[4] = dev_alloc(h, P * 4);
  p[5] = dev_alloc(h, P * 4); p[6] = dev_alloc(h, P * 4);
  p[7] = dev_alloc(h, sizeof(int64_t) * h->n_seg);
  p[8] = dev_alloc(h, sizeof(int32_t) * h->n_seg * 2);
  p[9] = dev_alloc(h, sizeof(int64_t) * (h->n_seg + 2));
  p[10] = dev_alloc(h, sizeof(Event) * (size_t)kEvCap * h->n_inst);
  p[11] = dev_alloc(h, sizeof(int64_t) * nodes * 2 + sizeof(double) * nodes + sizeof(float) * nodes);
  p[12] = dev_alloc(h, sizeof(InstConst) * h->n_inst);
  p[13] = dev_alloc(h, sizeof(InstDyn) * h->n_inst);
  // candidates per step: far above the expected P_cand * N (<= 1e-2 of all slots)
  const int64_t cand_cap = std::min<int64_t>(h->total_cap / 16 + 65536, 1LL << 30);
  p[14] = dev_alloc(h, sizeof(unsigned long long) * (size_t)cand_cap + 256);
  p[15] = dev_alloc(h, sizeof(PostScratch) * h->n_inst);
  for (int k = 0; k < 16; ++k)
    if (!p[k]) { pic_destroy(h); return PIC_ENOMEM; }
  st.z = (float*)p[0]; st.vx = (float*)p[1]; st.vy = (float*)p[2]; st.vz = (float*)p[3];
  st.id = (uint32_t*)p[4];
  st.dead_buf = (uint32_t*)p[5];
  st.dead_dense = (uint32_t*)p[6];
  st.seg_off = (const int64_t*)p[7];
  st.seg_cap = (const int32_t*)p[8];
  st.seg_count = (int32_t*)p[8] + h->n_seg;
  st.part = (int64_t*)p[9];
  st.ev_buf = (Event*)p[10];
  st.rho_acc = (int64_t*)p[11];
  st.rho = st.rho_acc + nodes;
  st.phi = (double*)(st.rho + nodes);
  st.E = (float*)(st.phi + nodes);
  st.ic = (const InstConst*)p[12];
  st.dyn = (InstDyn*)p[13];
  st.cand_cap = (int)cand_cap;
  st.cand_buf = (unsigned long long*)p[14];
  st.cand_count = (unsigned int*)((char*)p[14] + sizeof(unsigned long long) * (size_t)cand_cap);
  st.post = (PostScratch*)p[15];
  // counting-sort scratch: a second particle set plus histograms
  st.z2 = nullptr;
  cudaError_t e = cudaSuccess;
  e = cudaMemcpyAsync((void*)st.seg_off, h->seg_off.data(), sizeof(int64_t) * h->n_seg,
                      cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((void*)st.seg_cap, h->seg_cap.data(), sizeof(int32_t) * h->n_seg,
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(st.seg_count, 0, sizeof(int32_t) * h->n_seg, h->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(st.rho_acc, 0, sizeof(int64_t) * nodes * 2 + sizeof(double) * nodes +
                                           sizeof(float) * nodes, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((void*)st.ic, h->ic.data(), sizeof(InstConst) * h->n_inst,
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(st.dyn, 0, sizeof(InstDyn) * h->n_inst, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(st.part, 0, sizeof(int64_t) * (h->n_seg + 2), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(st.cand_count, 0, sizeof(unsigned int), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(st.post, 0, sizeof(PostScratch) * h->n_inst, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) { pic_destroy(h); return PIC_ECUDA; }
  int rc = set_launch_shape(h);
  if (rc != PIC_OK) { pic_destroy(h); return rc; }
  *out = h;
  return PIC_OK;
}

int pic_inject(pic_handle* h, int instance, int species, int64_t n, const float* z,
               const float* vx, const float* vy, const float* vz, int on_device) {
  if (!h || instance < 0 || instance >= h->n_inst || species < 0 || species > 2 || n < 0)
    return PIC_EINVAL;
  if (n == 0) return PIC_OK;
  if (!z || !vx || !vy || !vz) return PIC_EINVAL;
  const int g = 3 * instance + species;
  const float Lf = h->ic[instance].L_f;
  int32_t count = 0;
  InstDyn d;
  cudaError_t e = cudaMemcpyAsync(&count, h->st.seg_count + g, sizeof(int32_t),
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&d, h->st.dyn + instance, sizeof(InstDyn), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  if ((int64_t)count + n > h->seg_cap[g]) return PIC_ECAPACITY;
  if (!h->inject_flag) {
    h->inject_flag = (int*)dev_alloc(h, sizeof(int));
    if (!h->inject_flag) return PIC_ENOMEM;
  }
  // the particles go into the free slots after the live ones and their z
  // is checked there, on the device; they are counted in only if every z
  // lies in [0, L), so a rejected call leaves the instance as it was
  const int64_t base = h->seg_off[g] + count;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const size_t bytes = sizeof(float) * (size_t)n;
  e = cudaMemcpyAsync(h->st.z + base, z, bytes, kind, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->st.vx + base, vx, bytes, kind, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->st.vy + base, vy, bytes, kind, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->st.vz + base, vz, bytes, kind, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->inject_flag, 0, sizeof(int), h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  const unsigned blocks = (unsigned)((n + 255) / 256);
  k_count_outside<<<blocks, 256, 0, h->stream>>>(h->st.z + base, n, Lf, h->inject_flag);
  k_fill_ids<<<blocks, 256, 0, h->stream>>>(h->st.id + base, n, d.next_id);
  int hb = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&hb, h->inject_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  if (hb) return PIC_EINVAL;
  const int32_t newc = (int32_t)(count + n);
  const uint32_t nid = d.next_id + (uint32_t)n;
  e = cudaMemcpyAsync(h->st.seg_count + g, &newc, sizeof(int32_t), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h->st.dyn[instance].next_id, &nid, sizeof(uint32_t), cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  h->dirty = true;
  return PIC_OK;
}

int pic_set_step(pic_handle* h, int64_t step) {
  if (!h || step < 0) return PIC_EINVAL;
  std::vector<InstDyn> d(h->n_inst);
  cudaError_t e = cudaMemcpyAsync(d.data(), h->st.dyn, sizeof(InstDyn) * h->n_inst,
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  for (auto& x : d) x.step = step;
  e = cudaMemcpyAsync(h->st.dyn, d.data(), sizeof(InstDyn) * h->n_inst, cudaMemcpyHostToDevice,
                      h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  h->host_step = step;
  drop_graph(h);
  return PIC_OK;
}

// The plan of pic_step(n) from the current step: single steps up to a
// sort-aligned step (with a sort), graphs longest first, single steps for the
// rest.  With run set it launches the plan; otherwise it only captures the
// graphs the plan needs (pic_prepare_steps).
static int step_plan(pic_handle* h, int64_t n_steps, bool run) {
  int64_t left = n_steps, step = h->host_step;
  const int len = graph_unit(h);
  const int64_t sp = h->sort_period;
  // a graph bakes in where the periodic sort falls, so with a sort the graphs
  // start on sort-aligned steps: single steps up to the next aligned one
  if (len > 0 && sp > 0) {
    for (; left > 0 && step % sp != 0; --left, ++step) {
      if (!run) continue;
      cudaError_t e = launch_step(h);
      if (e != cudaSuccess) return cuda_fail_at(h, e, "step kernel launch");
    }
  }
  if (len > 0 && left > 0) {
    if (h->graphs.empty() || h->graphs[0].first != len) plan_graphs(h);
    // longest first: n steps run as floor(n / len) full graphs and the
    // binary digits of the rest (in sort periods when there is a sort)
    for (auto& g : h->graphs) {
      if (left >= g.first && !g.second) {
        int rc = build_graph(h, g.first, &g.second);
        if (rc != PIC_OK) return rc;
      }
      while (left >= g.first) {
        if (run) {
          cudaError_t e = cudaGraphLaunch(g.second, h->stream);
          if (e != cudaSuccess) return cuda_fail(h, e);
          h->host_step += g.first;
        }
        left -= g.first;
        step += g.first;
      }
    }
  }
  for (; run && left > 0; --left) {
    cudaError_t e = launch_step(h);
    if (e != cudaSuccess) return cuda_fail_at(h, e, "step kernel launch");
  }
  return run ? h->sticky : PIC_OK;
}

int pic_step(pic_handle* h, int64_t n_steps) {
  if (!h || n_steps < 0) return PIC_EINVAL;
  if (h->sticky != PIC_OK) return h->sticky;
  int rc = ensure_field(h);
  if (rc != PIC_OK) return rc;
  return step_plan(h, n_steps, true);
}

int pic_prepare_steps(pic_handle* h, int64_t n_steps) {
  if (!h || n_steps < 0) return PIC_EINVAL;
  if (h->sticky != PIC_OK) return h->sticky;
  int rc = ensure_field(h);
  if (rc != PIC_OK) return rc;
  return step_plan(h, n_steps, false);
}

int pic_profile_steps(pic_handle* h, int64_t n_steps, pic_profile* out) {
  if (!h || !out || n_steps < 0) return PIC_EINVAL;
  std::memset(out, 0, sizeof(*out));
  int rc = ensure_field(h);
  if (rc != PIC_OK) return rc;
  std::vector<cudaEvent_t> ev(6 * (size_t)std::max<int64_t>(n_steps, 1));
  for (auto& x : ev) cudaEventCreate(&x);
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  cudaEventRecord(t0, h->stream);
  std::vector<int> sorted(n_steps, 0);
  for (int64_t i = 0; i < n_steps; ++i) {
    cudaEvent_t* e = &ev[6 * i];
    cudaEventRecord(e[0], h->stream);
    push_kernel(h->push_chunk)<<<h->G, h->push_threads, h->push_smem, h->stream>>>(h->st);
    cudaEventRecord(e[1], h->stream);
    k_mid<<<mid_blocks(h), kPostThreads, h->mid_smem, h->stream>>>(h->st);
    cudaEventRecord(e[5], h->stream);
    k_post<<<3 * h->n_inst, kPostThreads, h->post_smem, h->stream>>>(h->st);
    launch_profile(h);
    cudaEventRecord(e[2], h->stream);
    h->host_step += 1;
    out->launches += h->st.prof_period > 0 ? 4 : 3;
    out->push_launches += 1;
    if (sort_due(h, h->host_step)) {
      cudaEventRecord(e[3], h->stream);
      launch_sort(h);
      cudaEventRecord(e[4], h->stream);
      sorted[i] = 1;
      out->launches += 3;
    }
  }
  cudaEventRecord(t1, h->stream);
  cudaError_t err = cudaEventSynchronize(t1);
  if (err == cudaSuccess) err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_fail(h, err);
  for (int64_t i = 0; i < n_steps; ++i) {
    float a = 0, b = 0, c = 0, m = 0;
    cudaEventElapsedTime(&a, ev[6 * i], ev[6 * i + 1]);
    cudaEventElapsedTime(&m, ev[6 * i + 1], ev[6 * i + 5]);
    cudaEventElapsedTime(&b, ev[6 * i + 5], ev[6 * i + 2]);
    out->ms_push += a;
    out->ms_mcc += m;
    out->ms_post += b;
    if (sorted[i]) {
      cudaEventElapsedTime(&c, ev[6 * i + 3], ev[6 * i + 4]);
      out->ms_sort += c;
    }
  }
  float tot = 0;
  cudaEventElapsedTime(&tot, t0, t1);
  out->ms_total = tot;
  out->steps = n_steps;
  for (auto& x : ev) cudaEventDestroy(x);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  return check_flags(h);
}

int pic_diagnostics(pic_handle* h, int instance, pic_diag* out) {
  if (!h || !out || instance < 0 || instance >= h->n_inst) return PIC_EINVAL;
  InstDyn d;
  int32_t counts[3];
  cudaError_t e = cudaMemcpyAsync(&d, h->st.dyn + instance, sizeof(InstDyn), cudaMemcpyDeviceToHost,
                                  h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(counts, h->st.seg_count + 3 * instance, sizeof(counts),
                        cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  fill_diag(h, instance, d, counts, out);
  return check_flags(h);
}

int pic_get_state(pic_handle* h, int instance, int species, float* z, float* vx, float* vy,
                  float* vz, uint32_t* id, int64_t cap, int64_t* n, int on_device) {
  if (!h || !n || instance < 0 || instance >= h->n_inst || species < 0 || species > 2)
    return PIC_EINVAL;
  const int g = 3 * instance + species;
  int32_t count = 0;
  cudaError_t e = cudaMemcpyAsync(&count, h->st.seg_count + g, sizeof(int32_t),
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  *n = count;
  if (cap < count) return PIC_ECAPACITY;
  const int64_t base = h->seg_off[g];
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t bytes = sizeof(float) * (size_t)count;
  if (count > 0) {
    if (z && e == cudaSuccess) e = cudaMemcpyAsync(z, h->st.z + base, bytes, kind, h->stream);
    if (vx && e == cudaSuccess) e = cudaMemcpyAsync(vx, h->st.vx + base, bytes, kind, h->stream);
    if (vy && e == cudaSuccess) e = cudaMemcpyAsync(vy, h->st.vy + base, bytes, kind, h->stream);
    if (vz && e == cudaSuccess) e = cudaMemcpyAsync(vz, h->st.vz + base, bytes, kind, h->stream);
    if (id && e == cudaSuccess) e = cudaMemcpyAsync(id, h->st.id + base, bytes, kind, h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  return check_flags(h);
}

int pic_get_rho_fixed(pic_handle* h, int instance, int64_t* out, int64_t n_nodes) {
  if (!h || !out || instance < 0 || instance >= h->n_inst) return PIC_EINVAL;
  const int nn = h->cfg[instance].n_cells + 1;
  if (n_nodes < nn) return PIC_EINVAL;
  int rc = ensure_field(h);
  if (rc != PIC_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(out, h->st.rho + h->ic[instance].node_off, sizeof(int64_t) * nn,
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  return check_flags(h);
}

int pic_get_field(pic_handle* h, int instance, double* phi, float* E, int64_t n_nodes) {
  if (!h || instance < 0 || instance >= h->n_inst) return PIC_EINVAL;
  const int nn = h->cfg[instance].n_cells + 1;
  if (n_nodes < nn) return PIC_EINVAL;
  int rc = ensure_field(h);
  if (rc != PIC_OK) return rc;
  const int off = h->ic[instance].node_off;
  // a step computes E only; phi of the current state is solved on request
  k_phi<<<h->n_inst, kPostThreads, h->field_smem, h->stream>>>(h->st);
  cudaError_t e = cudaGetLastError();
  if (phi && e == cudaSuccess)
    e = cudaMemcpyAsync(phi, h->st.phi + off, sizeof(double) * nn, cudaMemcpyDeviceToHost, h->stream);
  if (E && e == cudaSuccess)
    e = cudaMemcpyAsync(E, h->st.E + off, sizeof(float) * nn, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  return check_flags(h);
}

int pic_set_profile_period(pic_handle* h, int64_t period) {
  if (!h || period < 0) return PIC_EINVAL;
  if (h->sticky != PIC_OK) return h->sticky;
  const size_t tn = (size_t)h->total_nodes;
  const size_t bytes = sizeof(double) * tn + sizeof(long long) * 3 * tn + sizeof(long long) * h->n_inst;
  if (period > 0 && !h->st.phi_sum) {
    void* p = dev_alloc(h, bytes);
    if (!p) return PIC_ENOMEM;
    h->st.phi_sum = (double*)p;
    h->st.prof = (int64_t*)(h->st.phi_sum + tn);
    h->st.prof_n = h->st.prof + 3 * tn;
    h->st.tn = h->total_nodes;
  }
  if (h->st.phi_sum) {
    cudaError_t e = cudaMemsetAsync(h->st.phi_sum, 0, bytes, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
  }
  h->st.prof_period = period;
  drop_graph(h);
  return PIC_OK;
}

int pic_get_profiles(pic_handle* h, int instance, int64_t n_nodes, double* phi_avg,
                     double* density, int64_t* counts, int64_t* n_samples) {
  if (!h || instance < 0 || instance >= h->n_inst || !h->st.phi_sum) return PIC_EINVAL;
  const pic_config& c = h->cfg[instance];
  const int nn = c.n_cells + 1;
  if (n_nodes != nn) return PIC_EINVAL;
  const int off = h->ic[instance].node_off;
  std::vector<double> ps(nn);
  std::vector<long long> cnt(3 * (size_t)nn);
  long long K = 0;
  cudaError_t e = cudaMemcpyAsync(ps.data(), h->st.phi_sum + off, sizeof(double) * nn,
                                  cudaMemcpyDeviceToHost, h->stream);
  for (int sp = 0; sp < 3 && e == cudaSuccess; ++sp)
    e = cudaMemcpyAsync(cnt.data() + (size_t)sp * nn, h->st.prof + (size_t)sp * h->st.tn + off,
                        sizeof(long long) * nn, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&K, h->st.prof_n + instance, sizeof(long long), cudaMemcpyDeviceToHost,
                        h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  if (n_samples) *n_samples = K;
  if (counts)
    for (size_t i = 0; i < cnt.size(); ++i) counts[i] = cnt[i];
  const double nan = std::nan("");
  const double dz = c.gap_m / c.n_cells;
  if (phi_avg)
    for (int j = 0; j < nn; ++j) phi_avg[j] = K > 0 ? ps[j] / (double)K : nan;
  if (density)
    for (int sp = 0; sp < 3; ++sp)
      for (int j = 0; j < nn; ++j) {
        // linear weights of the node's particles over its length: dz inside,
        // dz/2 at the electrodes
        const double len = (j == 0 || j == nn - 1) ? 0.5 * dz : dz;
        density[(size_t)sp * nn + j] =
            K > 0 ? (double)cnt[(size_t)sp * nn + j] / (double)kTwo24 * c.weight / ((double)K * len) : nan;
      }
  return check_flags(h);
}

int pic_virtual_cathode(pic_handle* h, int instance, double near_fraction, pic_vc* out) {
  if (!h || !out || instance < 0 || instance >= h->n_inst || !(near_fraction > 0.0) ||
      near_fraction > 1.0)
    return PIC_EINVAL;
  const pic_config& c = h->cfg[instance];
  const int nn = c.n_cells + 1;
  std::vector<double> phi(nn);
  int64_t K = 0;
  int rc = pic_get_profiles(h, instance, nn, phi.data(), nullptr, nullptr, &K);
  if (rc != PIC_OK) return rc;
  if (K <= 0) return PIC_EINVAL;
  pic_diag d;
  rc = pic_diagnostics(h, instance, &d);
  if (rc != PIC_OK) return rc;
  std::memset(out, 0, sizeof(*out));
  out->samples = K;
  out->T_emit_eV = d.T_c_eV;
  out->net_efficiency = d.net_efficiency;
  // Eq. 10: the efficiency mapped to an equivalent barrier
  out->phi_vc_eff = d.net_efficiency > 0 ? d.T_c_eV * std::log(d.net_efficiency) : std::nan("");
  // near-cathode minimum of the averaged potential and its Eq. 9 transmission
  const int jmax = std::min(c.n_cells, std::max(1, (int)std::floor(near_fraction * c.n_cells)));
  int jm = 0;
  for (int j = 1; j <= jmax; ++j)
    if (phi[j] < phi[jm]) jm = j;
  out->phi_min = phi[jm];
  out->z_min = jm * (c.gap_m / c.n_cells);
  out->eta_vc = std::exp(out->phi_min / d.T_c_eV);
  return PIC_OK;
}

namespace {

struct CkptHeader {
  char magic[8];
  uint32_t abi, cfg_bytes, dyn_bytes, reserved;
  int32_t n_inst, n_seg, total_nodes, has_prof;
  int64_t prof_period, step;
};
const char kCkptMagic[8] = {'P', 'I', 'C', 'C', 'K', 'P', 'T', '1'};

// the fields that define a run: all but size, reserved0 and capacity
pic_config run_fields(pic_config c) {
  c.size = 0;
  c.reserved0 = 0;
  c.capacity[0] = c.capacity[1] = c.capacity[2] = 0;
  return c;
}

size_t ckpt_bytes(const pic_handle* h, const std::vector<int32_t>& counts, bool prof) {
  size_t b = sizeof(CkptHeader) + sizeof(pic_config) * h->n_inst + sizeof(int32_t) * 2 * h->n_seg +
             sizeof(InstDyn) * h->n_inst;
  for (int32_t n : counts) b += (size_t)n * 20;
  if (prof) b += sizeof(double) * h->total_nodes + sizeof(long long) * (3 * (size_t)h->total_nodes + h->n_inst);
  return b;
}

int read_counts(pic_handle* h, std::vector<int32_t>& counts) {
  counts.resize(h->n_seg);
  cudaError_t e = cudaMemcpyAsync(counts.data(), h->st.seg_count, sizeof(int32_t) * h->n_seg,
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? PIC_OK : cuda_fail(h, e);
}

}  // namespace

int pic_checkpoint_bytes(pic_handle* h, size_t* bytes) {
  if (!h || !bytes) return PIC_EINVAL;
  std::vector<int32_t> counts;
  int rc = read_counts(h, counts);
  if (rc != PIC_OK) return rc;
  *bytes = ckpt_bytes(h, counts, h->st.phi_sum != nullptr);
  return check_flags(h);
}

int pic_save(pic_handle* h, void* host_buf, size_t bytes, size_t* written) {
  if (!h || !host_buf) return PIC_EINVAL;
  if (h->sticky != PIC_OK) return h->sticky;
  std::vector<int32_t> counts;
  int rc = read_counts(h, counts);
  if (rc != PIC_OK) return rc;
  const bool prof = h->st.phi_sum != nullptr;
  const size_t need = ckpt_bytes(h, counts, prof);
  if (bytes < need) return PIC_ECAPACITY;
  std::vector<InstDyn> dyn(h->n_inst);
  cudaError_t e = cudaMemcpyAsync(dyn.data(), h->st.dyn, sizeof(InstDyn) * h->n_inst,
                                  cudaMemcpyDeviceToHost, h->stream);
  char* p = (char*)host_buf;
  CkptHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, kCkptMagic, 8);
  hd.abi = PIC_ABI_VERSION;
  hd.cfg_bytes = sizeof(pic_config);
  hd.dyn_bytes = sizeof(InstDyn);
  hd.n_inst = h->n_inst;
  hd.n_seg = h->n_seg;
  hd.total_nodes = h->total_nodes;
  hd.has_prof = prof ? 1 : 0;
  hd.prof_period = h->st.prof_period;
  hd.step = h->host_step;
  std::memcpy(p, &hd, sizeof(hd));
  p += sizeof(hd);
  std::memcpy(p, h->cfg.data(), sizeof(pic_config) * h->n_inst);
  p += sizeof(pic_config) * h->n_inst;
  std::memcpy(p, h->seg_cap.data(), sizeof(int32_t) * h->n_seg);
  p += sizeof(int32_t) * h->n_seg;
  std::memcpy(p, counts.data(), sizeof(int32_t) * h->n_seg);
  p += sizeof(int32_t) * h->n_seg;
  char* dyn_at = p;
  p += sizeof(InstDyn) * h->n_inst;
  for (int g = 0; g < h->n_seg && e == cudaSuccess; ++g) {
    const size_t n = (size_t)counts[g], b = 4 * n;
    const int64_t o = h->seg_off[g];
    if (n == 0) continue;
    e = cudaMemcpyAsync(p, h->st.z + o, b, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p + b, h->st.vx + o, b, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p + 2 * b, h->st.vy + o, b, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p + 3 * b, h->st.vz + o, b, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p + 4 * b, h->st.id + o, b, cudaMemcpyDeviceToHost, h->stream);
    p += 5 * b;
  }
  if (prof && e == cudaSuccess) {
    const size_t tn = (size_t)h->total_nodes;
    const size_t b = sizeof(double) * tn + sizeof(long long) * (3 * tn + h->n_inst);
    e = cudaMemcpyAsync(p, h->st.phi_sum, b, cudaMemcpyDeviceToHost, h->stream);
    p += b;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  std::memcpy(dyn_at, dyn.data(), sizeof(InstDyn) * h->n_inst);
  if (written) *written = (size_t)(p - (char*)host_buf);
  return check_flags(h);
}

int pic_load(pic_handle* h, const void* host_buf, size_t bytes) {
  if (!h || !host_buf || bytes < sizeof(CkptHeader)) return PIC_EINVAL;
  if (h->sticky != PIC_OK) return h->sticky;
  const char* p = (const char*)host_buf;
  const char* end = p + bytes;
  CkptHeader hd;
  std::memcpy(&hd, p, sizeof(hd));
  p += sizeof(hd);
  if (std::memcmp(hd.magic, kCkptMagic, 8) != 0 || hd.abi != PIC_ABI_VERSION ||
      hd.cfg_bytes != sizeof(pic_config) || hd.dyn_bytes != sizeof(InstDyn) ||
      hd.n_inst != h->n_inst || hd.n_seg != h->n_seg || hd.total_nodes != h->total_nodes ||
      hd.prof_period < 0 || hd.step < 0)
    return PIC_EINVAL;
  const size_t fixed = sizeof(pic_config) * h->n_inst + sizeof(int32_t) * 2 * h->n_seg +
                       sizeof(InstDyn) * h->n_inst;
  if ((size_t)(end - p) < fixed) return PIC_EINVAL;
  for (int i = 0; i < h->n_inst; ++i) {
    pic_config a, b = run_fields(h->cfg[i]);
    std::memcpy(&a, p + sizeof(pic_config) * i, sizeof(pic_config));
    a = run_fields(a);
    if (std::memcmp(&a, &b, sizeof(pic_config)) != 0) return PIC_EINVAL;
  }
  p += sizeof(pic_config) * h->n_inst;
  if (std::memcmp(p, h->seg_cap.data(), sizeof(int32_t) * h->n_seg) != 0) return PIC_EINVAL;
  p += sizeof(int32_t) * h->n_seg;
  std::vector<int32_t> counts(h->n_seg);
  std::memcpy(counts.data(), p, sizeof(int32_t) * h->n_seg);
  p += sizeof(int32_t) * h->n_seg;
  std::vector<InstDyn> dyn(h->n_inst);
  std::memcpy(dyn.data(), p, sizeof(InstDyn) * h->n_inst);
  p += sizeof(InstDyn) * h->n_inst;
  for (int g = 0; g < h->n_seg; ++g)
    if (counts[g] < 0 || counts[g] > h->seg_cap[g]) return PIC_EINVAL;
  for (const InstDyn& d : dyn)
    if (d.step != hd.step) return PIC_EINVAL;
  if (ckpt_bytes(h, counts, hd.has_prof != 0) > bytes) return PIC_EINVAL;
  // validated: from here on the handle takes the checkpoint's state
  if (hd.has_prof) {
    if (!h->st.phi_sum) {          // allocate the sums (overwritten below)
      int rc = pic_set_profile_period(h, 1);
      if (rc != PIC_OK) return rc;
    }
    h->st.prof_period = hd.prof_period;
  } else {
    int rc = pic_set_profile_period(h, 0);
    if (rc != PIC_OK) return rc;
  }
  cudaError_t e = cudaMemcpyAsync(h->st.seg_count, counts.data(), sizeof(int32_t) * h->n_seg,
                                  cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->st.dyn, dyn.data(), sizeof(InstDyn) * h->n_inst, cudaMemcpyHostToDevice,
                        h->stream);
  for (int g = 0; g < h->n_seg && e == cudaSuccess; ++g) {
    const size_t n = (size_t)counts[g], b = 4 * n;
    const int64_t o = h->seg_off[g];
    if (n == 0) continue;
    e = cudaMemcpyAsync(h->st.z + o, p, b, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->st.vx + o, p + b, b, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->st.vy + o, p + 2 * b, b, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->st.vz + o, p + 3 * b, b, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->st.id + o, p + 4 * b, b, cudaMemcpyHostToDevice, h->stream);
    p += 5 * b;
  }
  if (hd.has_prof && e == cudaSuccess) {
    const size_t tn = (size_t)h->total_nodes;
    const size_t b = sizeof(double) * tn + sizeof(long long) * (3 * tn + h->n_inst);
    e = cudaMemcpyAsync(h->st.phi_sum, p, b, cudaMemcpyHostToDevice, h->stream);
    p += b;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  h->host_step = hd.step;
  h->dirty = true;               // charge and field are recomputed from the particles
  drop_graph(h);
  return PIC_OK;
}

int pic_tune(pic_handle* h, const pic_tuning* t) {
  if (!h || !t || t->size != sizeof(pic_tuning)) return PIC_EINVAL;
  if (t->push_threads != 0) {
    if (t->push_threads < 64 || t->push_threads > 384 || t->push_threads % 32) return PIC_EINVAL;
    h->push_threads = t->push_threads;
    h->threads_set = true;
  }
  if (t->push_chunk != 0) {
    if (t->push_chunk != 32 && t->push_chunk != 64) return PIC_EINVAL;
    h->push_chunk = t->push_chunk;
    h->chunk_set = true;
  }
  if (t->push_blocks_per_sm != 0) {
    if (t->push_blocks_per_sm < 1 || t->push_blocks_per_sm > 32) return PIC_EINVAL;
    h->blocks_per_sm = t->push_blocks_per_sm;
  }
  if (t->sort_period != 0) h->sort_period = t->sort_period < 0 ? 0 : t->sort_period;
  h->st.agg = h->sort_period > 0 ? 1 : 0;
  if (t->graph_steps != 0) h->graph_steps = t->graph_steps < 0 ? 0 : t->graph_steps;
  if (t->wait_polls != 0) {
    if (t->wait_polls < -2) return PIC_EINVAL;
    h->st.wait_limit = t->wait_polls > 0 ? t->wait_polls : (t->wait_polls == -1 ? 0 : kWaitLimit);
  }
  if (h->sort_period > 0) {
    int rc = sort_alloc(h);
    if (rc != PIC_OK) return rc;
  }
  return set_launch_shape(h);
}

int pic_sort(pic_handle* h) {
  if (!h) return PIC_EINVAL;
  int rc = sort_alloc(h);
  if (rc != PIC_OK) return rc;
  launch_sort(h);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e);
  h->dirty = true;
  return PIC_OK;
}

const char* pic_last_error(const pic_handle* h) {
  if (!h) return "";
  return h->last_error;
}

int pic_synchronize(pic_handle* h) {
  if (!h) return PIC_EINVAL;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e);
  return check_flags(h);
}

void pic_destroy(pic_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_graph(h);
  free_all(h);
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

}  // extern "C"
