// pic_internal.cuh -- device-side state layout and helpers of the PIC-MCC
// library.  Internal to the library; the public boundary is include/pic.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pic {

constexpr int kMaxNz = 4096;          // shared-memory grid limit (nodes = Nz + 1)
constexpr int kMaxInstances = 1024;
constexpr int kEvCap = 2048;          // ionisation events per instance per step
constexpr int kPostThreads = 512;
constexpr int kMaxParts = 4;          // k_mid blocks per diode field / per segment list
constexpr int kHistMaxParticles = (1 << 20) - 256;
// push-block weights (shares of the particle range): nominal, bounds
constexpr int kNominalWeight = 1024, kMinWeight = 256, kMaxWeight = 4096;
constexpr int kWeightJumps = 8;    // weight updates that take the measured shares outright
// quads a push block bins before it flushes its histogram
constexpr int kSubQuads = kHistMaxParticles / 4;
constexpr long long kMaxSlots = 1LL << 29;            // particle slots per handle
constexpr int kDeadSmem = 8192;                       // absorbed slots staged in k_post
constexpr int kTwo24 = 1 << 24;

enum Tag : uint32_t { TAG_MCC = 1, TAG_EMIT = 2, TAG_EMIT_N = 3, TAG_REPL = 4 };
constexpr uint32_t kStreamInject = 3;

// sticky error bits: bit (-code - 1)
enum ErrBit : int32_t { ERR_CAPACITY = 1 << 3, ERR_TIMEOUT = 1 << 4, ERR_ENERGYCAP = 1 << 5 };

constexpr int kMccThreads = 256;

// Per-instance constants, derived on the host in FP64 and stored once.
struct InstConst {
  int32_t Nz;
  int32_t node_off;        // first node of this instance in the node arrays
  float inv_dz_f;          // (float)(Nz / L): the fixed-point cell rule multiplier
  float L_f;               // (float)L: absorbing-wall position
  float dt_f;
  float qmdt[3];           // q/m dt per species
  double dz, V, kappa;     // kappa = dz e w / (2^24 eps0): potential per fixed-point unit
  double inv_dz;
  double inv_nz;           // 1 / Nz
  // null-collision MCC
  uint32_t t_cand[3];      // candidate iff Philox word 0 < t_cand
  uint32_t key0[4];        // Philox4x32 key word 0 per stream (species 0..2, injection)
  uint32_t key1;
  uint32_t ckey[3];        // Philox2x32 candidate key per species
  float nu_max[3];
  float n_gas;
  float sig_n[3];          // neutral partner thermal speed sqrt(k T_n / M) per species
  float fm[3], fM[3];      // m/(m+M), M/(m+M)
  float half_mu_over_e[3]; // E_rel[eV] = this * g^2
  float two_e_over_mu[3];  // g^2 = this * E_rel[eV]
  float two_e_over_me;     // v^2 = this * E[eV] for electrons
  float sigma_el_e, sigma_cx_i, sigma_el_i;
  float E_exc, sigma_exc0, E_iz, lotz_aq;
  // injection (Sec. 2.1-2.2)
  int64_t emit_floor;
  uint32_t t_frac;
  float sig_w;             // sqrt(k T_w / m_e)
  float sig_e0, sig_i0;    // replenishment thermal speeds
  int32_t replenish;
  int32_t pad0;
  // diagnostics
  double weight;
  double m_d[3];
  int64_t window_start;
};

// Mutable per-instance state.
struct InstDyn {
  int64_t step;
  uint32_t next_id;
  int32_t ev_count;
  int32_t err;
  int32_t emit_dep;          // 1: a push block binned this step's emitted electrons
  int64_t win_steps;
  int64_t count[3][2];
  double ke[3][2];
  int64_t emitted;
  int64_t replenished;
  unsigned long long coll[6];
  unsigned long long cand[3];
  unsigned long long cap_exceeded;
  long long pushed;          // particle-steps since creation
};

// Hand-off from k_mid to the post kernel: absorbed counts, pre-compaction
// counts, the boundary tallies of the step, and the step number and first
// new id as they were when the step began (the post kernel closes the step
// in one of its blocks while the others still use them).
struct PostScratch {
  int D[3], N[3];
  uint32_t base_id;
  int32_t pad;
  long long step;
  long long cnt[3][kMaxParts][2];    // per species, per k_mid list block, per electrode
  double ke[3][kMaxParts][2];
};

struct Event {              // one ionisation: parent id + both children
  uint32_t parent;
  float z;
  float ve[3];
  float vi[3];
};

// Everything a kernel needs, passed by value.
struct DevState {
  int n_inst, n_seg;
  int G;                   // launched blocks of the particle kernels
  int W;                   // warps per block of the particle kernels
  int max_nodes;           // max (Nz + 1) over instances
  float* z; float* vx; float* vy; float* vz; uint32_t* id;
  float* z2; float* vx2; float* vy2; float* vz2; uint32_t* id2;   // sort scratch
  const int64_t* seg_off;  // [n_seg] first particle slot of each (instance, species)
  const int32_t* seg_cap;  // [n_seg]
  int32_t* seg_count;      // [n_seg] live particles
  int64_t* part;           // [n_seg + 2]: quad prefix of the last push, Q, G_eff
  int64_t* bstart;         // [G + 1]: first quad of each push block (b Q / G_eff)
  int32_t* dcount;         // [n_seg * G] absorbed particles per (segment, block)
  uint32_t* dead_buf;      // [total_cap] per-warp absorbed-slot lists (push), staging (post)
  uint32_t* dead_dense;    // [total_cap] per-block ordered absorbed-slot lists
  Event* ev_buf;           // [n_inst * kEvCap]
  int64_t* rho_acc;        // [total_nodes] fixed-point charge being accumulated
  int64_t* rho;            // [total_nodes] charge of the current state
  float* E;                // [total_nodes] field of the current state (FP32 copy)
  double* phi;             // [total_nodes]
  int32_t* sort_hist;      // counting-sort histograms, per segment [cell][chunk]
  const int64_t* sort_hoff;  // [n_seg] first histogram entry of each segment
  unsigned long long* cand_buf;  // [cand_cap] null-collision candidates: (segment << 32) | absolute slot
  unsigned int* cand_count;      // [1]
  int cand_cap;
  const InstConst* ic;
  InstDyn* dyn;
  PostScratch* post;       // [n_inst]
  // late-time profiles (sampled every prof_period steps of the window; 0 = off)
  long long prof_period;
  int tn;                  // total node slots over all instances (stride of prof)
  double* phi_sum;         // [tn] sum of sampled phi
  int64_t* prof;           // [3][tn] sum of sampled species deposits, 2^24 units per particle
  int64_t* prof_n;         // [n_inst] samples taken
  int wait_limit;          // polls of a push-kernel bulk-copy wait before PIC_ETIMEOUT
  int* bw;                 // [G] push-block weights: each block's share of the particles
  long long* bwp;          // [G + 1] their prefix sums in units of 2^-32 of the total (bwp[G] = 2^32)
  int* bt;                 // [G] streaming time of each block in the last push, ns
  int* bw_n;               // [1] weight updates since the last reset to equal shares
  int agg;
  int kp;                  // k_mid blocks per diode for its field, per segment for its lists
};

// Is the state after step n a profile sample?  (Sec. 3 late-time averages:
// steps n >= window_start with (n - window_start) a multiple of the period.)
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool profile_due(long long period, long long window_start, long long n) {
  return period > 0 && n >= window_start && (n - window_start) % period == 0;
}

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC'11.  Ten rounds of two 32x32->64 products with a Weyl-sequence key.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Philox2x32-10 word 0 (same paper): one 32x32->64 product per round on a
// 2-word counter, the ten round keys (key + r * 0x9E3779B9) precomputed.
// The per-particle null-collision candidate word.
__device__ __forceinline__ uint32_t philox2x32_w0_rk(uint32_t c0, uint32_t c1,
                                                     const uint32_t (&rk)[10]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p = (unsigned long long)0xD256D193u * c0;
    c0 = (uint32_t)(p >> 32) ^ rk[r] ^ c1;
    c1 = (uint32_t)p;
  }
  return c0;
}

// uniform on (0,1): (k + 1/2) 2^-23, k = r >> 9 -- exact in FP32
__device__ __forceinline__ float u01f(uint32_t r) {
  return (__uint2float_rn(r >> 9) + 0.5f) * 1.1920928955078125e-07f;
}

__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& n0, float& n1) {
  float rad = sqrtf(-2.0f * logf(u01f(a)));
  float s, c;
  sincospif(2.0f * u01f(b), &s, &c);
  n0 = rad * c;
  n1 = rad * s;
}

__device__ __forceinline__ void iso_dir(uint32_t rc, uint32_t rp, float& dx, float& dy, float& dz) {
  float c = 1.0f - 2.0f * u01f(rc);
  float s = sqrtf(fmaxf(0.0f, 1.0f - c * c));
  float sp, cp;
  sincospif(2.0f * u01f(rp), &sp, &cp);
  dx = s * cp;
  dy = s * sp;
  dz = c;
}

// Fixed-point cell rule, all FP32 round-to-nearest with no contraction:
// s = z * inv_dz, j = floor(s) clamped to [0, Nz-1], f = s - j.
// floor without a conversion: for 0 <= s < 2^22, s + 1.5*2^23 rounded toward
// zero is 1.5*2^23 + floor(s) (unit spacing there), read from its bits; the
// same sum less 1.5*2^23 is floor(s) as a float, exactly, so f needs no
// int-to-float conversion either.  A negative or NaN s (never a live
// particle) maps to a huge unsigned value and is clamped to the last cell, so
// every index stays in bounds.
__device__ __forceinline__ void cell_of(float z, float inv_dz, int Nz, int& j, float& f) {
  const float s = __fmul_rn(z, inv_dz);
  const float t = __fadd_rz(s, 12582912.0f);
  unsigned jj = (unsigned)(__float_as_int(t) - 0x4B400000);
  jj = min(jj, (unsigned)(Nz - 1));
  j = (int)jj;
  const float jf = fminf(__fsub_rn(t, 12582912.0f), (float)(Nz - 1));
  f = __fsub_rn(s, jf);
}

// Two FP32 values per instruction (the f32x2 forms of sm_100 and later):
// each element is rounded exactly like the scalar operation of the same
// rounding mode, so pairs give the scalar results bit for bit.
__device__ __forceinline__ unsigned long long f2_bits(float a, float b) {
  return ((unsigned long long)__float_as_uint(b) << 32) | (unsigned long long)__float_as_uint(a);
}
__device__ __forceinline__ void f2_split(unsigned long long u, float& a, float& b) {
  a = __uint_as_float((unsigned)u);
  b = __uint_as_float((unsigned)(u >> 32));
}
__device__ __forceinline__ unsigned long long mul2_rn(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long add2_rz(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long sub2_rn(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long fma2_rn(unsigned long long a, unsigned long long b,
                                                      unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// cell_of for two positions at once (same rule, same results)
__device__ __forceinline__ void cell_of2(float z0, float z1, float inv_dz, int Nz, int& j0,
                                         int& j1, float& f0, float& f1) {
  const unsigned long long s = mul2_rn(f2_bits(z0, z1), f2_bits(inv_dz, inv_dz));
  const unsigned long long t = add2_rz(s, f2_bits(12582912.0f, 12582912.0f));
  const unsigned long long tj = sub2_rn(t, f2_bits(12582912.0f, 12582912.0f));
  float t0, t1, a0, a1;
  f2_split(t, t0, t1);
  f2_split(tj, a0, a1);
  const unsigned top = (unsigned)(Nz - 1);
  j0 = (int)min((unsigned)(__float_as_int(t0) - 0x4B400000), top);
  j1 = (int)min((unsigned)(__float_as_int(t1) - 0x4B400000), top);
  const float ftop = (float)(Nz - 1);
  const unsigned long long f = sub2_rn(s, f2_bits(fminf(a0, ftop), fminf(a1, ftop)));
  f2_split(f, f0, f1);
}

// Q = trunc(f 2^24): f in [0, 1] makes the product exact and below 2^32, so a
// 32-bit conversion gives the rule's value (a 64-bit one would run on the
// FP64 pipe, which is narrow on this part).
__device__ __forceinline__ unsigned frac_units(float f) {
  return __float2uint_rz(__fmul_rn(f, 16777216.0f));
}

// ---------------------------------------------------------------- bulk copies
// 1D bulk copies global -> shared completing on an mbarrier (sm_90+ PTX).
// A warp streams its particles in chunks of cq quads (cq / 32 per lane),
// double-buffered in shared memory: 64 quads where the cell grid leaves room
// for ~24 resident warps per SM, 32 where it does not.
__host__ __device__ constexpr int stage_bytes(int cq) { return 3 * cq * 16; }  // (z, v_z, id)
constexpr int kWaitLimit = 1 << 20;   // bounded polls (each suspends up to kSuspendNs)
constexpr uint32_t kSuspendNs = 1000;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Test a phase; if it is not complete the warp is suspended (it issues
// nothing) until the phase completes or about kSuspendNs ns pass.
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0u;
}
// every wait ends: after kWaitLimit polls the caller gets false
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, uint32_t parity,
                                                  int limit = kWaitLimit) {
  for (int it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// ---------------------------------------------------------------- block scans
// Exclusive scan of one value per thread; *total gets the block sum.
// ws: shared scratch of >= 32 elements.  Must be called by all threads.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* total, T* ws) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T w = (lane < nw) ? ws[lane] : (T)0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    ws[lane] = w;
  }
  __syncthreads();
  T base = (wid > 0) ? ws[wid - 1] : (T)0;
  *total = ws[nw - 1];
  __syncthreads();
  return base + x - v;
}

// Exclusive scan of the first of two 64-bit values per thread and the block
// total of the second, in one pass.  ws: shared scratch of >= 32 elements.
// Must be called by all threads.
__device__ __forceinline__ void block_exclusive_scan_pair(long long x, long long y, long long* ex,
                                                          long long* ytot, long long* ws) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  long long a = x, b = y;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long pa = __shfl_up_sync(0xffffffffu, a, o);
    const long long pb = __shfl_up_sync(0xffffffffu, b, o);
    if (lane >= o) {
      a += pa;
      b += pb;
    }
  }
  __shared__ long long wsb[32];
  if (lane == 31) {
    ws[wid] = a;
    wsb[wid] = b;
  }
  __syncthreads();
  if (wid == 0) {
    long long wa = (lane < nw) ? ws[lane] : 0LL, wb = (lane < nw) ? wsb[lane] : 0LL;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long pa = __shfl_up_sync(0xffffffffu, wa, o);
      const long long pb = __shfl_up_sync(0xffffffffu, wb, o);
      if (lane >= o) {
        wa += pa;
        wb += pb;
      }
    }
    ws[lane] = wa;
    wsb[lane] = wb;
  }
  __syncthreads();
  *ex = ((wid > 0) ? ws[wid - 1] : 0LL) + a - x;
  *ytot = wsb[nw - 1];
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* ws) {
  T tot;
  (void)block_exclusive_scan<T>(v, &tot, ws);
  return tot;
}

}  // namespace pic
