// pic_kernels.cu -- sm_103a kernels of one PIC-MCC time step
// (arXiv 2605.07083, Sec. 2.1-2.2):
//
//   k_push    : gather E(z) from shared memory, leapfrog push (only v_z is
//               accelerated, 1D-3V), absorbing electrodes, the null-collision
//               candidate test on a Philox2x32 counter stream, and the
//               fixed-point charge deposit of the survivors into a per-block
//               shared-memory histogram flushed with 64-bit integer atomics.
//               One streaming pass over z, v_z, id, staged per warp by bulk
//               copies into shared memory.
//   k_mid     : the field of the new state, the ordered absorbed-slot lists
//               and boundary tallies, and the collisions of the step's
//               candidates, side by side.
//   k_post    : three blocks per diode, one per species: deterministic
//               hole-filling compaction, then the species' appends
//               (thermionic emission; ionisation children by parent id and
//               ion-loss replenishment); the ion block also closes the
//               diode's step.
//   k_field   : the Poisson/E solve alone (after a full deposit).
//   k_phi     : phi and E of the current state, on request.
//   k_profile : per-species density samples of the late-time profiles.
#include "pic_internal.cuh"

namespace pic {

// ------------------------------------------------------------------ partition
// Every particle kernel splits the concatenation of all (instance, species)
// segments, in units of 4 particles ("quads"), into G_eff contiguous ranges,
// one per block.  segS[g] = first quad of segment g, segS[n_seg] = total;
// segOff (when given) gets each segment's first slot, loaded in the same
// round trip.
__device__ void seg_quad_prefix(const DevState& st, long long* segS, long long* ws,
                                long long* segOff = nullptr) {
  long long carry = 0;
  for (int base = 0; base < st.n_seg; base += blockDim.x) {
    int g = base + threadIdx.x;
    if (segOff && g < st.n_seg) segOff[g] = st.seg_off[g];
    long long q = (g < st.n_seg) ? (long long)((st.seg_count[g] + 3) >> 2) : 0LL;
    long long tot;
    long long ex = block_exclusive_scan<long long>(q, &tot, ws);
    if (g < st.n_seg) segS[g] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) segS[st.n_seg] = carry;
  __syncthreads();
}

// blocks that get work: at least one quad per thread (the division only
// when fewer than grid * threads quads leave some blocks idle; Q is then
// below 2^31)
__device__ __forceinline__ int effective_blocks(long long Q, int grid, int threads) {
  if (Q > (long long)(grid - 1) * threads) return grid;
  const int need = (int)(((unsigned)Q + (unsigned)threads - 1u) / (unsigned)threads);
  return need < 1 ? 1 : need;
}

// floor(Q F / 2^32) for F <= 2^32, exactly (128-bit product); monotone in F
__device__ __forceinline__ long long scale_frac32(long long Q, unsigned long long F) {
  const unsigned long long q = (unsigned long long)Q;
  const unsigned long long lo = q * F, hi = __umul64hi(q, F);
  return (long long)((hi << 32) | (lo >> 32));
}

// quad range of warp w of a block range [q0, q1): contiguous, in warp order
// (a block range holds at most 2^18 quads, so 32-bit arithmetic is exact)
__device__ __forceinline__ long long warp_start(long long q0, long long q1, int w, int W) {
  return q0 + (long long)(((unsigned)(q1 - q0) * (unsigned)w) / (unsigned)W);
}

// ------------------------------------------------------------------ deposit
// Per-block charge histogram in shared memory with native 32-bit atomics.
// For cell j it keeps three counters side by side (one address, offsets 0,
// 4, 8): the particle count n, H = sum (Q >> 12) and L = sum Q mod 2^32 of
// the fixed-point fractions Q < 2^24.  A block bins fewer than 2^20
// particles (kHistMaxParticles), so H < 2^32 and the low parts R = sum
// (Q mod 2^12) < 2^32: sum Q = 2^12 H + R with R = (L - 2^12 H) mod 2^32,
// exact.  Node j's charge is then sign * (n_j 2^24 - Qs_j + Qs_{j-1}),
// Qs = sum Q -- exactly the linear-weight rule, in 64-bit integers at flush
// time.
struct Hist {
  unsigned* h3;              // [cell][count, sum Q >> 12, sum Q mod 2^32]
};

__device__ __forceinline__ void hist_zero(const Hist& h, int n_cells) {
  for (int j = threadIdx.x; j < 3 * n_cells; j += blockDim.x) h.h3[j] = 0u;
}

__device__ __forceinline__ long long qsum(const Hist& h, int j) {
  const unsigned H = h.h3[3 * j + 1], L = h.h3[3 * j + 2];
  return (long long)H * 4096 + (long long)(L - (H << 12));
}

// node charge of cells j-1 and j; callers sync before and after
__device__ __forceinline__ long long hist_node(const Hist& h, int j, int Nz) {
  long long v = 0;
  if (j < Nz) v += (long long)h.h3[3 * j] * kTwo24 - qsum(h, j);
  if (j > 0) v += qsum(h, j - 1);
  return v;
}

__device__ __forceinline__ void hist_flush(const Hist& h, int Nz, long long sgn, int64_t* dst) {
  for (int j = threadIdx.x; j <= Nz; j += blockDim.x) {
    const long long v = sgn * hist_node(h, j, Nz);
    if (v != 0) atomicAdd(reinterpret_cast<unsigned long long*>(dst + j), (unsigned long long)v);
  }
}

__device__ __forceinline__ void hist_add(const Hist& h, int j, unsigned q) {
  unsigned* c = h.h3 + 3 * j;
  atomicAdd(c, 1u);
  atomicAdd(c + 1, q >> 12);
  atomicAdd(c + 2, q);
}

// Deposit up to 4 particles per lane (bit k of am: z[k] is deposited).
// Called by all 32 lanes.  With agg set and the warp's cells spanning fewer
// than 4 cells (a state sorted by cell), the lanes bin in registers and the
// warp adds 12 totals; otherwise one set of atomics per particle.
__device__ __forceinline__ void deposit_warp(const Hist& h, const float (&z)[4], unsigned am,
                                             float inv_dz, int Nz, bool agg) {
  int j[4];
  unsigned q[4];
  int jlo = 0x7fffffff, jhi = -1;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    j[k] = 0;
    q[k] = 0u;
    if (am & (1u << k)) {
      float f;
      cell_of(z[k], inv_dz, Nz, j[k], f);
      q[k] = frac_units(f);
      jlo = min(jlo, j[k]);
      jhi = max(jhi, j[k]);
    }
  }
  if (agg) {
    const int wlo = __reduce_min_sync(0xffffffffu, jlo);
    const int whi = __reduce_max_sync(0xffffffffu, jhi);
    if (whi < 0) return;                        // nothing to deposit in this warp
    if (whi - wlo < 4) {
      unsigned c[4] = {0u, 0u, 0u, 0u}, hh[4] = {0u, 0u, 0u, 0u}, ll[4] = {0u, 0u, 0u, 0u};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (am & (1u << k)) {
          const int b = j[k] - wlo;
          const unsigned qh = q[k] >> 12, ql = q[k];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            c[t] += (b == t) ? 1u : 0u;
            hh[t] += (b == t) ? qh : 0u;
            ll[t] += (b == t) ? ql : 0u;
          }
        }
      }
      const int lane = threadIdx.x & 31;
      unsigned mine = 0u;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const unsigned sc = __reduce_add_sync(0xffffffffu, c[t]);
        const unsigned sh = __reduce_add_sync(0xffffffffu, hh[t]);
        const unsigned sl = __reduce_add_sync(0xffffffffu, ll[t]);
        if (lane == t) mine = sc;
        if (lane == 4 + t) mine = sh;
        if (lane == 8 + t) mine = sl;
      }
      // lane 4 w + t adds word w of cell wlo + t
      if (lane < 12 && mine != 0u) atomicAdd(h.h3 + 3 * (wlo + (lane & 3)) + (lane >> 2), mine);
      return;
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (am & (1u << k)) hist_add(h, j[k], q[k]);
}

// Deposit all four particles of every lane (none absorbed, no aggregation):
// straight-line code, the cell rule taken two particles at a time.
__device__ __forceinline__ void deposit_quad(const Hist& h, const float4& z4, float inv_dz,
                                             int Nz) {
  int j0, j1, j2, j3;
  float f0, f1, f2, f3;
  cell_of2(z4.x, z4.y, inv_dz, Nz, j0, j1, f0, f1);
  cell_of2(z4.z, z4.w, inv_dz, Nz, j2, j3, f2, f3);
  hist_add(h, j0, frac_units(f0));
  hist_add(h, j1, frac_units(f1));
  hist_add(h, j2, frac_units(f2));
  hist_add(h, j3, frac_units(f3));
}

// ------------------------------------------------------------------ MCC
// Null-collision Monte Carlo collision of one candidate (Sec. 2.2; Vahedi &
// Surendra).  Draw block 0: word 1 selects the process against the
// cumulative n sigma_k(E_rel) |g| (null beyond), words 2-3 the isotropic
// direction.  Block 1: neutral partner velocity (Maxwellian at T_n).  Block
// 2: ionisation energy split and the ejected electron's direction.
// Returns the new v_z; writes v_x, v_y in place.  Rare path: kept out of line.
__device__ __forceinline__ float collide(const InstConst* __restrict__ icg, InstDyn* dyn,
                                      Event* evb, float* vxp, float* vyp, int sp, uint32_t pid,
                                      uint32_t stepw, long long step, float z, float vz,
                                      int& code_out) {
  const InstConst& ic = *icg;
  const uint32_t k0 = ic.key0[sp], k1 = ic.key1;
  const uint4 A = philox10(make_uint4(pid, stepw, 0u, TAG_MCC), k0, k1);
  const uint4 B = philox10(make_uint4(pid, stepw, 1u, TAG_MCC), k0, k1);
  float n0, n1, n2, n3;
  box_muller(B.x, B.y, n0, n1);
  box_muller(B.z, B.w, n2, n3);
  const float sn = ic.sig_n[sp];
  const float vnx = sn * n0, vny = sn * n1, vnz = sn * n2;
  const float vx = *vxp, vy = *vyp;
  const float gx = vx - vnx, gy = vy - vny, gz = vz - vnz;
  const float g2 = gx * gx + gy * gy + gz * gz;
  const float gm = sqrtf(g2);
  const float Erel = ic.half_mu_over_e[sp] * g2;
  const float numax = ic.nu_max[sp];
  const float x = u01f(A.y) * numax;
  const bool in_win = step >= ic.window_start;
  const float fm = ic.fm[sp], fM = ic.fM[sp];
  float nvx = vx, nvy = vy, nvz = vz;
  int code = 0;
  if (sp < 2) {
    const float c0 = ic.n_gas * ic.sigma_el_e * gm;
    float sexc = 0.0f;
    if (ic.sigma_exc0 > 0.0f && Erel > ic.E_exc) sexc = ic.sigma_exc0 * (1.0f - ic.E_exc / Erel);
    const float c1 = c0 + ic.n_gas * sexc * gm;
    float siz = 0.0f;
    if (ic.lotz_aq > 0.0f && Erel > ic.E_iz) siz = ic.lotz_aq * logf(Erel / ic.E_iz) / (Erel * ic.E_iz);
    const float c2 = c1 + ic.n_gas * siz * gm;
    if (c2 > numax) {
      atomicOr(&dyn->err, ERR_ENERGYCAP);
      if (in_win) atomicAdd(&dyn->cap_exceeded, 1ull);
    }
    code = (x < c0) ? 1 : (x < c1) ? 2 : (x < c2) ? 3 : 0;
    if (code == 1 || code == 2) {
      float gn = gm;
      if (code == 2) gn = sqrtf((Erel - ic.E_exc) * ic.two_e_over_mu[sp]);
      float dx, dy, dz;
      iso_dir(A.z, A.w, dx, dy, dz);
      nvx = fm * vx + fM * vnx + fM * gn * dx;
      nvy = fm * vy + fM * vny + fM * gn * dy;
      nvz = fm * vz + fM * vnz + fM * gn * dz;
    } else if (code == 3) {
      const uint4 Cc = philox10(make_uint4(pid, stepw, 2u, TAG_MCC), k0, k1);
      const float Eex = Erel - ic.E_iz;
      const float U = u01f(Cc.x);
      const float E1 = U * Eex, E2 = (1.0f - U) * Eex;
      float d1x, d1y, d1z, d2x, d2y, d2z;
      iso_dir(A.z, A.w, d1x, d1y, d1z);
      iso_dir(Cc.y, Cc.z, d2x, d2y, d2z);
      const float s1 = sqrtf(E1 * ic.two_e_over_me), s2 = sqrtf(E2 * ic.two_e_over_me);
      nvx = vnx + s1 * d1x;
      nvy = vny + s1 * d1y;
      nvz = vnz + s1 * d1z;
      int slot = atomicAdd(&dyn->ev_count, 1);
      if (slot < kEvCap) {
        Event e;
        e.parent = pid;
        e.z = z;
        e.ve[0] = vnx + s2 * d2x;
        e.ve[1] = vny + s2 * d2y;
        e.ve[2] = vnz + s2 * d2z;
        e.vi[0] = vnx;
        e.vi[1] = vny;
        e.vi[2] = vnz;
        evb[slot] = e;
      } else {
        atomicOr(&dyn->err, ERR_CAPACITY);
      }
    }
  } else {
    const float c0 = ic.n_gas * ic.sigma_cx_i * gm;
    const float c1 = c0 + ic.n_gas * ic.sigma_el_i * gm;
    if (c1 > numax) {
      atomicOr(&dyn->err, ERR_ENERGYCAP);
      if (in_win) atomicAdd(&dyn->cap_exceeded, 1ull);
    }
    code = (x < c0) ? 4 : (x < c1) ? 5 : 0;
    if (code == 4) {            // charge exchange: the ion takes the neutral's velocity
      nvx = vnx;
      nvy = vny;
      nvz = vnz;
    } else if (code == 5) {
      float dx, dy, dz;
      iso_dir(A.z, A.w, dx, dy, dz);
      nvx = fm * vx + fM * vnx + fM * gm * dx;
      nvy = fm * vy + fM * vny + fM * gm * dy;
      nvz = fm * vz + fM * vnz + fM * gm * dz;
    }
  }
  code_out = code;
  if (code != 0) {
    *vxp = nvx;
    *vyp = nvy;
  }
  return nvz;
}

// The collisions of the step's null-collision candidates: thread t of a
// stride-`stride` team takes candidates t, t + stride, ...  A record is
// (segment << 32) | absolute slot; the thread's first record is read in the
// round trip of the count (a record at or past the count is never used, and
// the buffer holds cand_cap of them), so a candidate's particle is two round
// trips from the kernel's start.
__device__ void mcc_candidates(const DevState& st, unsigned t, unsigned stride) {
  const unsigned cap = (unsigned)st.cand_cap;
  const unsigned long long e_first = t < cap ? st.cand_buf[t] : 0ull;
  const unsigned n = min(*st.cand_count, cap);
  for (unsigned k = t; k < n; k += stride) {
    const unsigned long long e = k == t ? e_first : st.cand_buf[k];
    const int g = (int)(e >> 32);
    const long long slot = (long long)(e & 0xffffffffu);
    const int inst = g / 3, sp = g - 3 * inst;
    const long long step = st.dyn[inst].step;
    int code;
    const float vz = collide(st.ic + inst, st.dyn + inst, st.ev_buf + (long long)inst * kEvCap,
                             st.vx + slot, st.vy + slot, sp, st.id[slot], (uint32_t)step, step,
                             st.z[slot], st.vz[slot], code);
    st.vz[slot] = vz;
    if (step >= st.ic[inst].window_start) {
      // window tallies of candidates and outcomes: lanes with the same
      // (segment, outcome) add once -- one 64-bit atomic per candidate on a
      // handful of per-diode counters would serialise when candidates are
      // many (about 1 % of the particles per step at 40 V)
      const unsigned mask = __activemask();
      const unsigned peers = __match_any_sync(mask, ((unsigned)g << 3) | (unsigned)code);
      if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) {
        const unsigned long long c = (unsigned long long)__popc(peers);
        atomicAdd(&st.dyn[inst].cand[sp], c);
        atomicAdd(&st.dyn[inst].coll[code], c);
      }
    }
  }
}

// Thermionic electrons of a step (Sec. 2.2): how many (N = floor(x) + [r <
// frac(x)]) and electron k, a flux-weighted half-Maxwellian placed at z =
// v_z dt.  The field blocks (charge) and the electron blocks (the particles)
// both draw them, with the same arithmetic.
__device__ __forceinline__ int emitted_count(const InstConst& ic, long long step) {
  long long nem = ic.emit_floor;
  if (ic.t_frac != 0u) {
    const uint4 r = philox10(make_uint4(0u, (uint32_t)step, 0u, TAG_EMIT_N), ic.key0[kStreamInject],
                             ic.key1);
    if (r.x < ic.t_frac) nem += 1;
  }
  return (int)nem;
}

__device__ __forceinline__ void emitted_electron(const InstConst& ic, int k, long long step,
                                                 float& z, float& vx, float& vy, float& vz) {
  const uint4 r = philox10(make_uint4((uint32_t)k, (uint32_t)step, 0u, TAG_EMIT),
                           ic.key0[kStreamInject], ic.key1);
  float n0, n1;
  box_muller(r.x, r.y, n0, n1);
  vz = ic.sig_w * sqrtf(-2.0f * logf(u01f(r.z)));
  z = vz * ic.dt_f;
  vx = ic.sig_w * n0;
  vy = ic.sig_w * n1;
}

// ------------------------------------------------------------------ k_push
struct SegCtx {
  float inv_dz, Lf, dt, qmdt;
  int Nz;
  uint32_t tc, ck, stepw;
  uint32_t rk[10];          // Philox2x32 round keys of the candidate stream
};

// One particle: gather, leapfrog, wall test and the null-collision candidate
// test.  Returns bit 0 = absorbed, bit 1 = collision candidate (its
// collision is applied afterwards by k_mid; it changes velocities only, so
// the survivor's z is final here and is deposited by the caller).
// Es2[j] = (E_j, E_{j+1} - E_j): one 64-bit shared load per gather
__device__ __forceinline__ unsigned push_one(const SegCtx& c, const float2* Es2,
                                             float& z, float& vz, uint32_t pid) {
  int j;
  float f;
  cell_of(z, c.inv_dz, c.Nz, j, f);
  const float2 e = Es2[j];
  const float Ez = fmaf(f, e.y, e.x);
  vz = fmaf(c.qmdt, Ez, vz);
  z = fmaf(vz, c.dt, z);
  if (!(z >= 0.0f && z < c.Lf)) return 1u;
  if (c.tc != 0u && philox2x32_w0_rk(pid, c.stepw, c.rk) < c.tc) return 2u;
  return 0u;
}

// Four particles of one lane, with no data-dependent branch: the gathers,
// pushes and the four Philox2x32 chains are independent and interleave.  The
// candidate word is computed for absorbed particles too and masked off.
__device__ __forceinline__ void push_quad(const SegCtx& c, const float2* Es2, float4& z4,
                                          float4& v4, const uint4& id4, unsigned& dm,
                                          unsigned& cm) {
  float z[4] = {z4.x, z4.y, z4.z, z4.w};
  float v[4] = {v4.x, v4.y, v4.z, v4.w};
  const uint32_t id[4] = {id4.x, id4.y, id4.z, id4.w};
  unsigned d = 0u;
  int j[4];
  float f[4];
  cell_of2(z[0], z[1], c.inv_dz, c.Nz, j[0], j[1], f[0], f[1]);
  cell_of2(z[2], z[3], c.inv_dz, c.Nz, j[2], j[3], f[2], f[3]);
  float Ez[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 e = Es2[j[k]];
    Ez[k] = fmaf(f[k], e.y, e.x);
  }
  // v += (q/m dt) E, z += v dt, two particles per instruction
  const unsigned long long qm2 = f2_bits(c.qmdt, c.qmdt), dt2 = f2_bits(c.dt, c.dt);
#pragma unroll
  for (int k = 0; k < 4; k += 2) {
    const unsigned long long v2 = fma2_rn(qm2, f2_bits(Ez[k], Ez[k + 1]), f2_bits(v[k], v[k + 1]));
    const unsigned long long z2 = fma2_rn(v2, dt2, f2_bits(z[k], z[k + 1]));
    f2_split(v2, v[k], v[k + 1]);
    f2_split(z2, z[k], z[k + 1]);
  }
  // wall test of the quad at once: for the bits of z + 0 (the sum turns -0
  // into +0 and leaves every other value, NaN included, as it is),
  // 0 <= z < L is an unsigned compare with the bits of L; only a quad with
  // a particle outside tests each particle
  {
    const unsigned long long zero2 = f2_bits(0.0f, 0.0f);
    float y0, y1, y2, y3;
    f2_split(add2_rz(f2_bits(z[0], z[1]), zero2), y0, y1);
    f2_split(add2_rz(f2_bits(z[2], z[3]), zero2), y2, y3);
    const unsigned hi = max(max(__float_as_uint(y0), __float_as_uint(y1)),
                            max(__float_as_uint(y2), __float_as_uint(y3)));
    if (hi >= __float_as_uint(c.Lf)) {
#pragma unroll
      for (int k = 0; k < 4; ++k) d |= (z[k] >= 0.0f && z[k] < c.Lf) ? 0u : (1u << k);
    }
  }
  unsigned m = 0u;
  if (c.tc != 0u) {                      // uniform over the segment
    uint32_t a[4], b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      a[k] = id[k];
      b[k] = c.stepw;
    }
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const unsigned long long p = (unsigned long long)0xD256D193u * a[k];
        a[k] = (uint32_t)(p >> 32) ^ c.rk[r] ^ b[k];
        b[k] = (uint32_t)p;
      }
    }
    // candidates are rare: test the quad's smallest word first
    if (min(min(a[0], a[1]), min(a[2], a[3])) < c.tc) {
#pragma unroll
      for (int k = 0; k < 4; ++k) m |= (a[k] < c.tc) ? (1u << k) : 0u;
      m &= ~d;
    }
  }
  z4 = make_float4(z[0], z[1], z[2], z[3]);
  v4 = make_float4(v[0], v[1], v[2], v[3]);
  dm = d;
  cm = m;
}

// The field of one diode into shared memory as (E_j, E_{j+1} - E_j) pairs,
// j < Nz, with up to kU loads of each kind in flight per thread: a plain
// loop waits for one L2 round trip per iteration (six at 2048 cells and 384
// threads, ~1 us of every push block's start).
__device__ __forceinline__ void stage_field(float2* Es2, const float* __restrict__ Eg, int Nz,
                                            int j_begin = 0) {
  constexpr int kU = 8;
  for (int base = j_begin; base < Nz; base += kU * (int)blockDim.x) {
    float e0[kU], e1[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int j = base + u * (int)blockDim.x + (int)threadIdx.x;
      e0[u] = j < Nz ? __ldg(Eg + j) : 0.0f;
      e1[u] = j < Nz ? __ldg(Eg + j + 1) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int j = base + u * (int)blockDim.x + (int)threadIdx.x;
      if (j < Nz) Es2[j] = make_float2(e0[u], e1[u] - e0[u]);
    }
  }
}

// Chunk ch of a warp's quads [wq0, wq1) of a segment at slot off: its z,
// v_z and id into stage ch & 1 of the warp, completing on that stage's
// mbarrier.  Issued by one lane.
template <int CQ>
__device__ __forceinline__ void issue_chunk(const DevState& st, unsigned char* wstage,
                                            unsigned long long* wbar, long long off, int wq0,
                                            int wq1, int ch) {
  constexpr int kChunkQuads = CQ, kArrBytes = CQ * 16, kStageBytes = stage_bytes(CQ);
  const int s = ch & 1;
  const int qc = wq0 + kChunkQuads * ch;
  const int nq = (wq1 - qc) < kChunkQuads ? (wq1 - qc) : kChunkQuads;
  const uint32_t bytes = (uint32_t)nq * 16u;
  unsigned char* b = wstage + s * kStageBytes;
  const long long at = off + 4LL * qc;
  fence_proxy_async();
  mbar_expect_tx(&wbar[s], 3u * bytes);
  bulk_g2s(b, st.z + at, bytes, &wbar[s]);
  bulk_g2s(b + kArrBytes, st.vz + at, bytes, &wbar[s]);
  bulk_g2s(b + 2 * kArrBytes, st.id + at, bytes, &wbar[s]);
}

// Wait for stage s of the warp's chunk ch.  If the copy does not complete in
// time: flag it, let this warp's copies in flight (this stage and the next)
// land with the full limit, keep the stage parities in step and return
// false, so that the warp stops its part of the segment.
__device__ __forceinline__ bool stage_ready(const DevState& st, unsigned long long* wbar,
                                            unsigned& phase, int s, int ch, int nchunks,
                                            int inst, int lane) {
  const bool arrived = mbar_wait_bounded(&wbar[s], (phase >> s) & 1u, st.wait_limit);
  if (!__all_sync(0xffffffffu, arrived)) {
    if (lane == 0) atomicOr(&st.dyn[inst].err, ERR_TIMEOUT);
    if (mbar_wait_bounded(&wbar[s], (phase >> s) & 1u)) phase ^= 1u << s;
    if (ch + 1 < nchunks && mbar_wait_bounded(&wbar[s ^ 1], (phase >> (s ^ 1)) & 1u))
      phase ^= 1u << (s ^ 1);
    return false;
  }
  phase ^= 1u << s;
  return true;
}

// Collision candidates -> the compact global list (one atomic per warp);
// absorbed slots -> this warp's ordered list (warp scans).  Called by all 32
// lanes for a chunk in which some lane has either; q is the lane's quad.
__device__ __forceinline__ void record_events(const DevState& st, int g, int inst, long long off,
                                              int q, unsigned cm, unsigned dm, uint32_t* dbuf,
                                              int& dead_run, int lane) {
  const int cc = __popc(cm), dc = __popc(dm);
  int ci = cc, di = dc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int yc = __shfl_up_sync(0xffffffffu, ci, o);
    const int yd = __shfl_up_sync(0xffffffffu, di, o);
    if (lane >= o) { ci += yc; di += yd; }
  }
  const int ctot = __shfl_sync(0xffffffffu, ci, 31);
  const int dtot = __shfl_sync(0xffffffffu, di, 31);
  if (ctot) {
    unsigned cbase = 0;
    if (lane == 0) cbase = atomicAdd(st.cand_count, (unsigned)ctot);
    cbase = __shfl_sync(0xffffffffu, cbase, 0);
    unsigned w = cbase + (unsigned)(ci - cc);
    for (int k2 = 0; k2 < 4; ++k2) {
      if (cm & (1u << k2)) {
        if (w < (unsigned)st.cand_cap)
          st.cand_buf[w] = ((unsigned long long)g << 32) | (unsigned long long)(off + 4 * q + k2);
        else
          atomicOr(&st.dyn[inst].err, ERR_CAPACITY);
        ++w;
      }
    }
  }
  if (dtot) {
    int w = dead_run + di - dc;
    for (int k2 = 0; k2 < 4; ++k2)
      if (dm & (1u << k2)) dbuf[w++] = (uint32_t)(4 * q + k2);
    dead_run += dtot;
  }
}

template <bool kDepositOnly, int CQ>
__device__ __forceinline__ void push_body(const DevState& st) {
  constexpr int kChunkQuads = CQ, kArrBytes = CQ * 16, kStageBytes = stage_bytes(CQ);
  static_assert(CQ % 32 == 0 && CQ <= 128, "whole quads per lane");
  extern __shared__ __align__(16) unsigned char smem[];
  const int mn = st.max_nodes;
  float2* Es2 = reinterpret_cast<float2*>(smem);
  Hist hist;
  hist.h3 = reinterpret_cast<unsigned*>(smem + (size_t)mn * 8);
  long long* segS = reinterpret_cast<long long*>(smem + (size_t)mn * 20 + ((mn & 1) ? 4 : 0));
  long long* segOff = segS + st.n_seg + 1;
  // per-warp double-buffered staging of (z, v_z, id) chunks and their mbarriers
  const size_t stage_off =
      ((size_t)mn * 20 + 8 + (size_t)(2 * st.n_seg + 1) * 8 + 127) & ~(size_t)127;
  unsigned char* stages = smem + stage_off;
  unsigned long long* bars =
      reinterpret_cast<unsigned long long*>(stages + (size_t)(blockDim.x >> 5) * 2 * kStageBytes);
  __shared__ long long ws64[32];
  __shared__ int wcount[32];
  __shared__ InstConst icS;

  if (!kDepositOnly && (threadIdx.x & 31) == 0) {
    mbar_init(&bars[2 * (threadIdx.x >> 5)], 1u);
    mbar_init(&bars[2 * (threadIdx.x >> 5) + 1], 1u);
    fence_mbar_init();
  }
  // A handle of one diode: every block works on instance 0 (node offset 0,
  // Nz = max_nodes - 1), so its constants and the first kPre * blockDim.x
  // field pairs are loaded before the partition is known, in the round trip
  // of the segment counts.
  constexpr int kPre = 8;
  const bool pre = !kDepositOnly && st.n_inst == 1;
  constexpr int kIcWords = (int)(sizeof(InstConst) / 4);
  int icw = 0;
  float pe0[kPre], pe1[kPre];
  if (pre) {
    if ((int)threadIdx.x < kIcWords) icw = __ldg(reinterpret_cast<const int*>(st.ic) + threadIdx.x);
    const int nz = st.max_nodes - 1;
#pragma unroll
    for (int u = 0; u < kPre; ++u) {
      const int j = u * (int)blockDim.x + (int)threadIdx.x;
      pe0[u] = j < nz ? __ldg(st.E + j) : 0.0f;
      pe1[u] = j < nz ? __ldg(st.E + j + 1) : 0.0f;
    }
  }
  // the block's weight prefix is read in the same round trip as the segment
  // counts and offsets (the total is wG unless fewer blocks get work)
  unsigned long long w0 = 0, w1 = 0;
  if (!kDepositOnly && threadIdx.x == 0) {
    w0 = (unsigned long long)st.bwp[blockIdx.x];
    w1 = (unsigned long long)st.bwp[blockIdx.x + 1];
  }
  seg_quad_prefix(st, segS, ws64, segOff);
  const long long Q = segS[st.n_seg];
  // One thread finds the block's range and the barrier hands it on (64-bit
  // divisions here, a long software sequence in every thread, held each
  // block ~1.7 us; the full grid's path below has none).
  __shared__ long long range_s[2];
  __shared__ int geff_s;
  if (threadIdx.x == 0) {
    const int Geff = effective_blocks(Q, gridDim.x, blockDim.x);
    long long lo = 0, hi = 0;
    if ((int)blockIdx.x < Geff) {
      if (kDepositOnly) {
        lo = (long long)blockIdx.x * Q / Geff;
        hi = ((long long)blockIdx.x + 1) * Q / Geff;
      } else {
        // the block's share of the quads is its weight (integer, set from
        // each block's throughput in the last push, so that SMs that stream
        // slower get less and all blocks finish together).  bwp holds the
        // weights' prefix sums as fractions of their total in units of
        // 2^-32 (bwp[0] = 0, bwp[G] = 2^32), and the ranges are exact
        // integer functions of it, monotone, so they tile [0, Q) exactly.
        // When fewer than the launched blocks get work (a state of fewer
        // quads than threads), the first G_eff blocks share it by their
        // part of the prefix.
        if (Geff == (int)gridDim.x) {
          lo = scale_frac32(Q, w0);
          hi = scale_frac32(Q, w1);
        } else {
          const unsigned long long tot = (unsigned long long)st.bwp[Geff];
          lo = (long long)((unsigned long long)Q * w0 / tot);
          hi = (long long)((unsigned long long)Q * w1 / tot);
        }
        // the block ranges, for the post kernel (which would otherwise
        // redo G_eff 64-bit divisions on one SM)
        st.bstart[blockIdx.x] = lo;
        if ((int)blockIdx.x == Geff - 1) st.bstart[Geff] = hi;
      }
    }
    range_s[0] = lo;
    range_s[1] = hi;
    geff_s = Geff;
  }
  __syncthreads();
  const int Geff = geff_s;
  const long long lo = range_s[0], hi = range_s[1];
  if (!kDepositOnly && blockIdx.x == 0) {
    for (int g = threadIdx.x; g <= st.n_seg; g += blockDim.x) st.part[g] = segS[g];
    if (threadIdx.x == 0) st.part[st.n_seg + 1] = Geff;
    // the ionisation events of this step are counted from zero (k_mid
    // appends them, the post kernel reads the count)
    for (int i = threadIdx.x; i < st.n_inst; i += blockDim.x) st.dyn[i].ev_count = 0;
  }
  if ((int)blockIdx.x >= Geff) return;
  if (lo >= hi) {
    if (!kDepositOnly && threadIdx.x == 0) st.bt[blockIdx.x] = 0;
    return;
  }
  int cur = -1;
  if (pre) {
    // instance 0's constants and field from the registers loaded above; the
    // barrier at the start of the segment loop publishes them
    const int nz = st.max_nodes - 1;
    int* dst = reinterpret_cast<int*>(&icS);
    if ((int)threadIdx.x < kIcWords) dst[threadIdx.x] = icw;
    for (int w = threadIdx.x + blockDim.x; w < kIcWords; w += blockDim.x)
      dst[w] = reinterpret_cast<const int*>(st.ic)[w];
#pragma unroll
    for (int u = 0; u < kPre; ++u) {
      const int j = u * (int)blockDim.x + (int)threadIdx.x;
      if (j < nz) Es2[j] = make_float2(pe0[u], pe1[u] - pe0[u]);
    }
    stage_field(Es2, st.E, nz, kPre * (int)blockDim.x);
    cur = 0;
  }
  const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // first segment whose quad range ends after lo
  int glo = 0, ghi = st.n_seg - 1;
  while (glo < ghi) {
    int mid = (glo + ghi) >> 1;
    if (segS[mid + 1] > lo) ghi = mid; else glo = mid + 1;
  }

  unsigned phase = 0u;                 // parity of this warp's two stage barriers
  unsigned char* wstage = stages + (size_t)warp * 2 * kStageBytes;
  unsigned long long* wbar = bars + 2 * warp;
  const unsigned long long t_start = global_ns();
  for (int g = glo; g < st.n_seg && segS[g] < hi; ++g) {
    const long long s0 = segS[g], s1 = segS[g + 1];
    if (s1 <= lo || s1 == s0) continue;
    const int inst = g / 3, sp = g - 3 * inst;
    const long long sgn = (sp == 2) ? 1LL : -1LL;
    __syncthreads();
    // quads of this block, relative to the segment: 32-bit (a segment holds
    // < 2^31 particles); taken kSubQuads at a time, each sub-range binned
    // and flushed on its own so that no counter of the histogram overflows
    const int q0 = (int)((lo > s0 ? lo : s0) - s0);
    const int q1 = (int)((hi < s1 ? hi : s1) - s0);
    const long long off = segOff[g];
    if (!kDepositOnly && lane == 0) {
      // the warp's first two chunks are in flight while the block stages
      // the diode's constants and field
      const int b0 = (q1 - q0 > kSubQuads) ? q0 + kSubQuads : q1;
      const int pw0 = (int)warp_start(q0, b0, warp, W), pw1 = (int)warp_start(q0, b0, warp + 1, W);
      if (pw1 > pw0) issue_chunk<CQ>(st, wstage, wbar, off, pw0, pw1, 0);
      if (pw1 - pw0 > kChunkQuads) issue_chunk<CQ>(st, wstage, wbar, off, pw0, pw1, 1);
    }
    if (inst != cur) {
      // the diode's constants, and its field read with the node offset and
      // cell count each thread loads itself, so that the field's loads go
      // out in the round trip after the constants' (hist_zero below reads
      // icS after the barrier)
      const InstConst* icg = st.ic + inst;
      const int* src = reinterpret_cast<const int*>(icg);
      int* dst = reinterpret_cast<int*>(&icS);
      for (int w = threadIdx.x; w < kIcWords; w += blockDim.x) dst[w] = src[w];
      if (!kDepositOnly) stage_field(Es2, st.E + __ldg(&icg->node_off), __ldg(&icg->Nz));
      __syncthreads();
      cur = inst;
    }
    int dead_total = 0;                // absorbed slots the block listed for this segment
    for (int a = q0; a < q1; a += kSubQuads) {
      const int b1 = (q1 - a > kSubQuads) ? a + kSubQuads : q1;
      hist_zero(hist, icS.Nz);
      __syncthreads();
      if (!kDepositOnly && sp < 2 && a == 0 && s0 == segS[3 * inst]) {
        // this block holds the diode's first particle, an electron: it also
        // bins the charge of the electrons the step emits (Sec. 2.2), so the
        // field of the new state needs nothing more than the push's charge
        const long long step = st.dyn[inst].step;
        const int Nemit = emitted_count(icS, step);
        for (int base = 0; base < Nemit; base += blockDim.x) {
          const int k = base + threadIdx.x;
          float ze[4] = {0.0f, 0.0f, 0.0f, 0.0f};
          unsigned am = 0u;
          if (k < Nemit) {
            float vx, vy, vz;
            emitted_electron(icS, k, step, ze[0], vx, vy, vz);
            am = 1u;
          }
          deposit_warp(hist, ze, am, icS.inv_dz_f, icS.Nz, true);
        }
        if (threadIdx.x == 0) st.dyn[inst].emit_dep = 1;
      }
      const int wq0 = (int)warp_start(a, b1, warp, W), wq1 = (int)warp_start(a, b1, warp + 1, W);
      const int N = st.seg_count[g];
      float* __restrict__ zp = st.z + off;
      float* __restrict__ vzp = st.vz + off;
      const float inv_dz = icS.inv_dz_f;
      const int Nz = icS.Nz;
      const bool agg = st.agg != 0;

      SegCtx c;
      c.inv_dz = inv_dz;
      c.Lf = icS.L_f;
      c.dt = icS.dt_f;
      c.qmdt = icS.qmdt[sp];
      c.Nz = Nz;
      c.tc = icS.t_cand[sp];
      c.ck = icS.ckey[sp];
      c.stepw = kDepositOnly ? 0u : (uint32_t)st.dyn[inst].step;
  #pragma unroll
      for (int r = 0; r < 10; ++r) c.rk[r] = c.ck + (uint32_t)r * 0x9E3779B9u;
      uint32_t* dbuf = st.dead_buf + off + 4 * wq0;
      int dead_run = 0;

      // chunk ch of this warp = quads [wq0 + kChunkQuads ch, +kChunkQuads), two
      // per lane; bulk copies run two chunks ahead of the compute
      const int nchunks = (wq1 - wq0 + kChunkQuads - 1) / kChunkQuads;
      if (!kDepositOnly && lane == 0 && a != q0) {   // the first sub-range's are issued
        if (nchunks > 0) issue_chunk<CQ>(st, wstage, wbar, off, wq0, wq1, 0);
        if (nchunks > 1) issue_chunk<CQ>(st, wstage, wbar, off, wq0, wq1, 1);
      }
      int ch = 0;
      bool stop = false;
      if (!kDepositOnly) {
        // the warp's leading chunks that hold only live particles: each
        // lane reads its two quads, the stage is refilled with chunk ch + 2,
        // then straight-line push and (unless one of the warp's particles
        // left the gap or the state is sorted) deposit
        const int live_end = min(wq1, N >> 2);
        const int nfull = live_end > wq0 ? (live_end - wq0) / kChunkQuads : 0;
        for (; ch < nfull; ++ch) {
          const int s = ch & 1;
          if (!stage_ready(st, wbar, phase, s, ch, nchunks, inst, lane)) {
            stop = true;
            break;
          }
          const unsigned char* b = wstage + s * kStageBytes;
          constexpr int kSub = kChunkQuads / 32;  // quads per lane
          float4 zA[kSub], vA[kSub];
          uint4 iA[kSub];
#pragma unroll
          for (int h = 0; h < kSub; ++h) {
            const int o = 512 * h + 16 * lane;
            zA[h] = *reinterpret_cast<const float4*>(b + o);
            vA[h] = *reinterpret_cast<const float4*>(b + kArrBytes + o);
            iA[h] = *reinterpret_cast<const uint4*>(b + 2 * kArrBytes + o);
          }
          __syncwarp();
          if (lane == 0 && ch + 2 < nchunks) issue_chunk<CQ>(st, wstage, wbar, off, wq0, wq1, ch + 2);
#pragma unroll
          for (int h = 0; h < kSub; ++h) {
            float4 z4 = zA[h], v4 = vA[h];
            unsigned dm, cm;
            push_quad(c, Es2, z4, v4, iA[h], dm, cm);
            const int q = wq0 + kChunkQuads * ch + 32 * h + lane;
            __stcs(reinterpret_cast<float4*>(zp + 4 * q), z4);
            __stcs(reinterpret_cast<float4*>(vzp + 4 * q), v4);
            // one vote: most quads of a warp have no absorbed particle and
            // no candidate
            const bool evt = __any_sync(0xffffffffu, (cm | dm) != 0u);
            if (!evt && !agg) {
              deposit_quad(hist, z4, inv_dz, Nz);
            } else {
              const float zz[4] = {z4.x, z4.y, z4.z, z4.w};
              deposit_warp(hist, zz, ~dm & 0xFu, inv_dz, Nz, agg);
              if (evt) record_events(st, g, inst, off, q, cm, dm, dbuf, dead_run, lane);
            }
          }
        }
      }
      // the rest: a chunk that ends the warp's range or holds the segment's
      // last (partial) quad, one particle at a time; k_deposit takes all of
      // its chunks here
      for (; !stop && ch < nchunks; ++ch) {
        const unsigned char* b = nullptr;
        if (!kDepositOnly) {
          const int s = ch & 1;
          if (!stage_ready(st, wbar, phase, s, ch, nchunks, inst, lane)) break;
          b = wstage + s * kStageBytes;
        }
        for (int h = 0; h < kChunkQuads / 32; ++h) {
          const int q = wq0 + kChunkQuads * ch + 32 * h + lane;
          unsigned dm = 0, cm = 0, am = 0;
          float zz[4] = {0.0f, 0.0f, 0.0f, 0.0f};
          if (q < wq1) {
            const int i = 4 * q;
            float4 z4s = make_float4(0.f, 0.f, 0.f, 0.f), v4s = z4s;
            uint4 id4s = make_uint4(0u, 0u, 0u, 0u);
            if (!kDepositOnly) {
              const int o = 512 * h + 16 * lane;
              z4s = *reinterpret_cast<const float4*>(b + o);
              v4s = *reinterpret_cast<const float4*>(b + kArrBytes + o);
              id4s = *reinterpret_cast<const uint4*>(b + 2 * kArrBytes + o);
            }
            const float zq[4] = {z4s.x, z4s.y, z4s.z, z4s.w};
            const float vq[4] = {v4s.x, v4s.y, v4s.z, v4s.w};
            const uint32_t iq[4] = {id4s.x, id4s.y, id4s.z, id4s.w};
            for (int k2 = 0; k2 < 4; ++k2) {
              if (i + k2 < N) {
                float zv = kDepositOnly ? zp[i + k2] : zq[k2];
                if (!kDepositOnly) {
                  float vv = vq[k2];
                  const unsigned r = push_one(c, Es2, zv, vv, iq[k2]);
                  if (r & 1u) dm |= 1u << k2;
                  if (r & 2u) cm |= 1u << k2;
                  zp[i + k2] = zv;
                  vzp[i + k2] = vv;
                }
                if (!(dm & (1u << k2))) {
                  zz[k2] = zv;
                  am |= 1u << k2;
                }
              }
            }
          }
          deposit_warp(hist, zz, am, inv_dz, Nz, agg);
          if (!kDepositOnly && __any_sync(0xffffffffu, (cm | dm) != 0u))
            record_events(st, g, inst, off, q, cm, dm, dbuf, dead_run, lane);
        }
        if (!kDepositOnly) {
          __syncwarp();
          if (lane == 0 && ch + 2 < nchunks) issue_chunk<CQ>(st, wstage, wbar, off, wq0, wq1, ch + 2);
        }
      }
      // concatenate the warps' ordered lists into one list per block
      if (!kDepositOnly) {
        if (lane == 0) wcount[warp] = dead_run;
        __syncthreads();
        int start = 0, total = 0;
        for (int w = 0; w < W; ++w) {
          if (w < warp) start += wcount[w];
          total += wcount[w];
        }
        uint32_t* dst = st.dead_dense + off + 4 * q0 + dead_total + start;
        for (int k2 = lane; k2 < dead_run; k2 += 32) dst[k2] = dbuf[k2];
        dead_total += total;
        if (threadIdx.x == 0) st.dcount[(long long)g * st.G + blockIdx.x] = dead_total;
      }
      __syncthreads();
      hist_flush(hist, Nz, sgn, st.rho_acc + icS.node_off);
    }
  }
  if (!kDepositOnly && threadIdx.x == 0)
    st.bt[blockIdx.x] = (int)min(global_ns() - t_start, 2000000000ull);
}

// the push with 64-quad and with 32-quad warp chunks
__global__ void __launch_bounds__(384, 2) k_push(DevState st) { push_body<false, 64>(st); }
__global__ void __launch_bounds__(384, 2) k_push32(DevState st) { push_body<false, 32>(st); }
__global__ void k_deposit(DevState st) { push_body<true, 64>(st); }

// ------------------------------------------------------------------ field solve
// Poisson with Dirichlet phi_0 = 0, phi_Nz = V (Sec. 2.1), solved exactly by
// summation: with d_j = phi_{j+1} - phi_j the difference equations give
// d_j = d_0 - kappa G_j, G_j = sum_{k=1..j} rho_k (exact int64), and
// phi_Nz = V fixes d_0 = (V + kappa sum_{j<Nz} G_j) / Nz.  E_j = -(d_j +
// d_{j-1}) / (2 dz) inside, one-sided at the electrodes.  phi_j = j d_0 -
// kappa sum_{k<j} G_k is written only when phi is non-null: the push needs E
// alone, and FP64 work is scarce on this part.  rho_s is the block's shared
// copy of the fixed-point charge; it is overwritten with G.  Only nodes in
// [jlo, jhi) are written: the integer scans are cheap, so several blocks can
// each solve the whole system and share the FP64 work of writing E.
__device__ void field_solve(const InstConst& ic, long long* rho_s, float* E, double* phi,
                            long long* ws, int jlo = 0, int jhi = 1 << 30) {
  const int Nz = ic.Nz;
  const int nt = blockDim.x;
  const int c = (Nz + nt - 1) / nt;            // <= 8 for Nz <= 4096, nt = 512
  const int j0 = threadIdx.x * c;
  long long a[8];
  long long loc = 0, wl = 0;                   // sum rho_k; sum rho_k (Nz - k)
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    if (u < c) {
      const int j = j0 + u;
      const long long v = (j >= 1 && j < Nz) ? rho_s[j] : 0LL;
      loc += v;
      wl += v * (long long)(Nz - j);
      a[u] = loc;
    }
  }
  // one scan of the pair: the exclusive prefix of loc is G at the node
  // before this thread's first; the total of wl is sum_{j < Nz} G_j
  long long ex, Htot;
  block_exclusive_scan_pair(loc, wl, &ex, &Htot, ws);
  // E_j = -(d_j + d_{j-1}) / (2 dz) = A + B (G_j + G_{j-1}),  A = -d0/dz, B = kappa/(2 dz);
  // one warp evaluates the constants (FP64 units are few per SM)
  __shared__ double dAB[3];
  const double kap = ic.kappa;
  if (threadIdx.x < 32) {
    const double d0w = (ic.V + kap * (double)Htot) * ic.inv_nz;
    if (threadIdx.x == 0) {
      dAB[0] = d0w;
      dAB[1] = -d0w * ic.inv_dz;
      dAB[2] = 0.5 * kap * ic.inv_dz;
    }
  }
  __syncthreads();
  const double d0 = dAB[0], A = dAB[1], B = dAB[2];
  long long gprev = ex;                        // G_{j0 - 1}
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int j = j0 + u;
    if (u < c && j < Nz) {
      const long long gj = ex + a[u];
      const long long gsum = (j == 0) ? 0LL : gj + gprev;
      if (j >= jlo && j < jhi) E[j] = (float)fma(B, (double)gsum, A);
      gprev = gj;
      a[u] = gj;
    }
  }
  if (j0 < Nz && j0 + c >= Nz && Nz >= jlo && Nz < jhi)
    E[Nz] = (float)fma(2.0 * B, (double)gprev, A);                           // G_{Nz-1}
  if (phi) {
    // phi_j = j d0 - kappa sum_{k<j} G_k: a second scan, for sampled or
    // requested potentials only
    long long lsum = 0, hx[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (u < c && j0 + u < Nz) {
        hx[u] = lsum;
        lsum += a[u];
      }
    long long tot;
    const long long hex = block_exclusive_scan<long long>(lsum, &tot, ws);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int j = j0 + u;
      if (u < c && j < Nz && j >= jlo && j < jhi)
        phi[j] = fma((double)j, d0, -kap * (double)(hex + hx[u]));
    }
    if (threadIdx.x == 0 && Nz >= jlo && Nz < jhi) phi[Nz] = ic.V;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kPostThreads) k_field(DevState st) {
  extern __shared__ __align__(16) unsigned char smem[];
  long long* rho_s = reinterpret_cast<long long*>(smem);
  __shared__ long long ws64[32];
  const InstConst& ic = st.ic[blockIdx.x];
  const int nn = ic.Nz + 1;
  const int off = ic.node_off;
  for (int j = threadIdx.x; j < nn; j += blockDim.x) {
    const long long v = st.rho_acc[off + j];
    rho_s[j] = v;
    st.rho[off + j] = v;
    st.rho_acc[off + j] = 0;
  }
  __syncthreads();
  field_solve(ic, rho_s, st.E + off, st.phi + off, ws64);
}

// phi (and E, identically) of the current state from its fixed-point charge,
// for callers that read the potential; a time step computes E only.
__global__ void __launch_bounds__(kPostThreads) k_phi(DevState st) {
  extern __shared__ __align__(16) unsigned char smem[];
  long long* rho_s = reinterpret_cast<long long*>(smem);
  __shared__ long long ws64[32];
  const InstConst& ic = st.ic[blockIdx.x];
  const int nn = ic.Nz + 1;
  const int off = ic.node_off;
  for (int j = threadIdx.x; j < nn; j += blockDim.x) rho_s[j] = st.rho[off + j];
  __syncthreads();
  field_solve(ic, rho_s, st.E + off, st.phi + off, ws64);
}

// ------------------------------------------------------------------ weights
// New push-block weights from the last push: block b streamed its share w_b
// in t_b ns, so its rate is w_b / t_b; the next shares follow the rates
// (relative to their mean), halfway from the old weights, within
// [kMinWeight, kMaxWeight].  Blocks without a time keep their weight.  Then
// the prefix sums over all launched blocks.  One block does it; every block
// of the next push reads the result.
__device__ void update_push_weights(const DevState& st, int G, float* ws, long long* ws64) {
  float r_sum = 0.0f, n = 0.0f;
  for (int b = threadIdx.x; b < G; b += blockDim.x) {
    const int t = st.bt[b];
    if (t > 0) {
      r_sum += (float)st.bw[b] / (float)t;
      n += 1.0f;
    }
  }
  r_sum = block_sum<float>(r_sum, ws);
  n = block_sum<float>(n, ws);
  if (n <= 0.0f || !(r_sum > 0.0f)) return;
  const float mean = r_sum / n;
  // the first updates after a reset jump to the measured shares; later ones
  // move halfway, which damps the step-to-step noise of the block times
  const int n_upd = *st.bw_n;
  const float keep = n_upd < kWeightJumps ? 0.0f : 0.5f;
  for (int b = threadIdx.x; b < G; b += blockDim.x) {
    const int t = st.bt[b];
    if (t <= 0) continue;
    const float target = (float)kNominalWeight * ((float)st.bw[b] / (float)t) / mean;
    const float w = keep * (float)st.bw[b] + (1.0f - keep) * target;
    st.bw[b] = (int)fminf(fmaxf(rintf(w), (float)kMinWeight), (float)kMaxWeight);
  }
  __syncthreads();
  // The prefix as fractions of the total in units of 2^-32 (the push turns
  // them into quad ranges with a multiply).  Any map of the prefix that is
  // monotone, 0 at 0 and 2^32 at the total tiles the quads exactly; a float
  // scale is one (rounding keeps order), clamped, with the total's entry
  // set exactly.  With one pass (G <= blockDim.x) the raw prefix stays in a
  // register; otherwise each thread rescales the entries it wrote.
  const bool one_pass = st.G <= (int)blockDim.x;
  long long carry = 0, mine = 0;
  for (int base = 0; base < st.G; base += blockDim.x) {
    const int b = base + threadIdx.x;
    const long long w = b < st.G ? (long long)st.bw[b] : 0LL;
    long long tot;
    const long long ex = block_exclusive_scan<long long>(w, &tot, ws64);
    if (b < st.G) {
      if (one_pass) mine = carry + ex + w;
      else st.bwp[b + 1] = carry + ex + w;
    }
    carry += tot;
  }
  const float scale = 4294967296.0f / (float)carry;
  for (int b = threadIdx.x; b < st.G; b += blockDim.x) {
    const long long P = one_pass ? mine : st.bwp[b + 1];
    const long long F = (long long)((float)P * scale);
    st.bwp[b + 1] = b + 1 == st.G ? (1LL << 32) : (F < (1LL << 32) ? F : (1LL << 32));
  }
  if (threadIdx.x == 0) {
    st.bwp[0] = 0;
    if (n_upd < kWeightJumps) *st.bw_n = n_upd + 1;
  }
}

// ------------------------------------------------------------------ k_mid / k_post
// After the push the step finishes in two kernels.
//
// k_mid, three kinds of blocks working side by side:
//   * per diode, the charge and field of the new state: the survivors'
//     charge k_push left in rho_acc plus that of the electrons emitted this
//     step (ionisation children and replenished pairs are an electron and an
//     ion at one position, so their charge is zero node by node), then E;
//   * per (diode, species), the ordered list of the step's absorbed slots
//     and the boundary tallies of Sec. 2.3 (counts, FP64 kinetic energy);
//   * the collisions of the null-collision candidates (MCC).
// k_post, per (diode, species): deterministic hole filling, then the
// species' appends (thermionic electrons; ionisation children ordered by
// parent id; replenished pairs); the ion block closes the diode's step.

__device__ __forceinline__ void put_particle(const DevState& st, long long off, long long slot,
                                             float z, float vx, float vy, float vz, uint32_t id) {
  st.z[off + slot] = z;
  st.vx[off + slot] = vx;
  st.vy[off + slot] = vy;
  st.vz[off + slot] = vz;
  st.id[off + slot] = id;
}

// sum of (c0, c1, e0, e1) over the block, fixed order; valid in thread 0.
// The FP64 adds (slow on this part: a few FP64 lanes per SM) run only in
// warps that hold a non-zero energy; adding the zeros would give the same
// sums.
__device__ __forceinline__ void block_reduce4(long long& c0, long long& c1, double& e0, double& e1,
                                              long long* wsl, double* wsd) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c0 += __shfl_down_sync(0xffffffffu, c0, o);
    c1 += __shfl_down_sync(0xffffffffu, c1, o);
  }
  if (__any_sync(0xffffffffu, e0 != 0.0 || e1 != 0.0)) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e0 += __shfl_down_sync(0xffffffffu, e0, o);
      e1 += __shfl_down_sync(0xffffffffu, e1, o);
    }
  }
  if (lane == 0) {
    wsl[wid] = c0;
    wsl[32 + wid] = c1;
    wsd[wid] = e0;
    wsd[32 + wid] = e1;
  }
  __syncthreads();
  if (wid == 0) {
    c0 = lane < nw ? wsl[lane] : 0LL;
    c1 = lane < nw ? wsl[32 + lane] : 0LL;
    e0 = lane < nw ? wsd[lane] : 0.0;
    e1 = lane < nw ? wsd[32 + lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      c0 += __shfl_down_sync(0xffffffffu, c0, o);
      c1 += __shfl_down_sync(0xffffffffu, c1, o);
    }
    if (__any_sync(0xffffffffu, e0 != 0.0 || e1 != 0.0)) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        e0 += __shfl_down_sync(0xffffffffu, e0, o);
        e1 += __shfl_down_sync(0xffffffffu, e1, o);
      }
    }
  }
  __syncthreads();
}

// Ionisation events of the step ordered by parent id: keys (parent << 32 | k)
// in evk[0, P2), bitonic sort in shared memory.
__device__ void sort_events(const Event* evb, int E, unsigned long long* evk) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (E <= 1) {
    if (E == 1 && tid == 0) evk[0] = 0ull;
    __syncthreads();
    return;
  }
  int P2 = 1;
  while (P2 < E) P2 <<= 1;
  for (int k = tid; k < P2; k += nt)
    evk[k] = (k < E) ? (((unsigned long long)evb[k].parent << 32) | (unsigned)k) : ~0ull;
  __syncthreads();
  for (int kk = 2; kk <= P2; kk <<= 1) {
    for (int jj = kk >> 1; jj > 0; jj >>= 1) {
      for (int i = tid; i < P2; i += nt) {
        const int ixj = i ^ jj;
        if (ixj > i) {
          const unsigned long long a = evk[i], b = evk[ixj];
          const bool up = (i & kk) == 0;
          if ((a > b) == up) { evk[i] = b; evk[ixj] = a; }
        }
      }
      __syncthreads();
    }
  }
}

// Field of the new state of one diode (k_mid).
__device__ void mid_field(const DevState& st, int inst, int part, unsigned char* smem,
                          long long* ws64) {
  __shared__ InstConst ic;
  __shared__ int sNemit;
  __shared__ long long sStep;
  const int tid = threadIdx.x, nt = blockDim.x;
  const InstConst* icg = st.ic + inst;
  // a handle of one diode has node offset 0 and max_nodes nodes: its charge
  // loads need not wait for the constants
  const bool one = st.n_inst == 1;
  const int nn = one ? st.max_nodes : icg->Nz + 1, off = one ? 0 : icg->node_off;
  {
    const int* src = reinterpret_cast<const int*>(icg);
    int* dst = reinterpret_cast<int*>(&ic);
    for (int w = tid; w < (int)(sizeof(InstConst) / 4); w += nt) dst[w] = src[w];
  }
  // the push's charge (k_post clears rho_acc once every part has read it),
  // up to kU loads per thread in flight
  long long* rho_s = reinterpret_cast<long long*>(smem);            // [nn]
  const int64_t* acc = st.rho_acc + off;
  constexpr int kU = 8;
  for (int base = 0; base < nn; base += kU * nt) {
    long long v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int j = base + u * nt + tid;
      v[u] = j < nn ? acc[j] : 0LL;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int j = base + u * nt + tid;
      if (j < nn) rho_s[j] = v[u];
    }
  }
  if (tid == 0) {
    const long long step = st.dyn[inst].step;
    sStep = step;
    sNemit = st.dyn[inst].emit_dep ? 0 : emitted_count(*icg, step);
    if (part == 0) {
      PostScratch* ps = st.post + inst;
      ps->step = step;
      ps->base_id = st.dyn[inst].next_id;
    }
  }
  __syncthreads();
  const long long step = sStep;
  const int Nemit = sNemit;
  if (Nemit > 0) {
    // no push block binned this step's emitted electrons (the diode has no
    // electron in flight): their charge is added here
    Hist h;
    h.h3 = reinterpret_cast<unsigned*>(rho_s + nn);
    hist_zero(h, ic.Nz);
    __syncthreads();
    for (int base = 0; base < Nemit; base += nt) {
      const int k = base + tid;
      float zz[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      unsigned am = 0u;
      if (k < Nemit) {
        float vx, vy, vz;
        emitted_electron(ic, k, step, zz[0], vx, vy, vz);
        am = 1u;
      }
      deposit_warp(h, zz, am, ic.inv_dz_f, ic.Nz, true);
    }
    __syncthreads();
    for (int j = tid; j < nn; j += nt) rho_s[j] -= hist_node(h, j, ic.Nz);
    __syncthreads();
  }
  if (part == 0)
    for (int j = tid; j < nn; j += nt) st.rho[off + j] = rho_s[j];
  const int jlo = (int)((long long)part * nn / st.kp);
  const int jhi = (int)((long long)(part + 1) * nn / st.kp);
  const bool sample = profile_due(st.prof_period, ic.window_start, step);
  field_solve(ic, rho_s, st.E + off, sample ? st.phi + off : nullptr, ws64, jlo, jhi);
  if (sample) {
    double* pa = st.phi_sum + off;
    const double* ph = st.phi + off;
    for (int j = jlo + tid; j < jhi; j += nt) pa[j] += ph[j];
    if (part == 0 && tid == 0) st.prof_n[inst] += 1;
  }
}

// The ordered list of segment g's absorbed slots (the push blocks' lists
// concatenated in block order, which is slot order) and its boundary
// tallies.  kp blocks per segment: each finds the whole block prefix and
// takes the list entries k = part + kp (tid + nt i), so the FP64 kinetic
// energies are spread over kp SMs; the post kernel adds the parts' sums in
// part order.
__device__ void mid_absorbed(const DevState& st, int g, int part, unsigned char* smem,
                             int* ws32, long long* wsl, double* wsd) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int inst = g / 3, sp = g - 3 * inst;
  const int G = st.G, kp = st.kp;
  long long* blo = reinterpret_cast<long long*>(smem);               // [G + 1]
  int* bpre = reinterpret_cast<int*>(blo + G + 1);                   // [G + 1]
  // one round trip: block starts and absorbed counts of every launched
  // block (only those of blocks with work are used), and the segment's
  // numbers
  for (int b = tid; b <= G; b += nt) {
    blo[b] = st.bstart[b];
    bpre[b] = b < G ? st.dcount[(long long)g * G + b] : 0;
  }
  const int Geff = (int)st.part[st.n_seg + 1];
  const long long off = st.seg_off[g];
  const int N = st.seg_count[g];
  const long long Sg = st.part[g];
  const long long qg = (N + 3) >> 2;
  __syncthreads();
  int carry = 0;
  for (int base = 0; base < Geff; base += nt) {
    const int b = base + tid;
    int c = 0;
    if (b < Geff) {
      const long long lb = blo[b], hb = blo[b + 1];
      if (qg > 0 && lb < hb && lb < Sg + qg && hb > Sg) c = bpre[b];
    }
    __syncthreads();                   // bpre is overwritten with the prefix below
    int tot;
    const int ex = block_exclusive_scan<int>(c, &tot, ws32);
    if (b < Geff) bpre[b] = carry + ex;
    carry += tot;
  }
  if (tid == 0) bpre[Geff] = carry;
  __syncthreads();
  const int D = carry;
  uint32_t* dd = st.dead_buf + off;
  const InstConst& ic = st.ic[inst];
  const double mw = 0.5 * ic.m_d[sp] * ic.weight;
  long long cnt0 = 0, cnt1 = 0;
  double ke0 = 0.0, ke1 = 0.0;
  for (int k = part + kp * tid; k < D; k += kp * nt) {
    int blo_i = 0, bhi_i = Geff;
    while (bhi_i - blo_i > 1) {
      const int mid = (blo_i + bhi_i) >> 1;
      if (bpre[mid] <= k) blo_i = mid; else bhi_i = mid;
    }
    const long long lb = blo[blo_i];
    const long long q0b = (lb > Sg ? lb : Sg) - Sg;
    const uint32_t idx = st.dead_dense[off + 4 * q0b + (k - bpre[blo_i])];
    dd[k] = idx;
    const float z = st.z[off + idx];
    const double vx = st.vx[off + idx], vy = st.vy[off + idx], vz = st.vz[off + idx];
    const double ke = mw * (vx * vx + vy * vy + vz * vz);
    if (z < 0.0f) { cnt0 += 1; ke0 += ke; } else { cnt1 += 1; ke1 += ke; }
  }
  block_reduce4(cnt0, cnt1, ke0, ke1, wsl, wsd);
  if (tid == 0) {
    PostScratch* ps = st.post + inst;
    if (part == 0) {
      ps->D[sp] = D;
      ps->N[sp] = N;
    }
    ps->cnt[sp][part][0] = cnt0;
    ps->cnt[sp][part][1] = cnt1;
    ps->ke[sp][part][0] = ke0;
    ps->ke[sp][part][1] = ke1;
  }
}

// Blocks [0, n_inst): field of diode b.  [n_inst, 4 n_inst): absorbed list
// and tallies of segment b - n_inst.  Block 4 n_inst: re-weights the push
// blocks for the next step.  The rest: the candidates' collisions.
__global__ void __launch_bounds__(kPostThreads, 2) k_mid(DevState st) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long wsl[64];
  __shared__ double wsd[64];
  __shared__ long long ws64[32];
  __shared__ int ws32[32];
  const int b = blockIdx.x, kp = st.kp, nf = st.n_inst * kp;
  if (b < nf) {
    mid_field(st, b / kp, b % kp, smem, ws64);
  } else if (b < 4 * nf) {
    mid_absorbed(st, (b - nf) / kp, (b - nf) % kp, smem, ws32, wsl, wsd);
  } else if (b == 4 * nf) {
    update_push_weights(st, (int)st.part[st.n_seg + 1], reinterpret_cast<float*>(wsd), ws64);
  } else {
    // candidate k goes to block k mod nb, so the collisions' arithmetic is
    // spread over every collision block's SM
    const unsigned m = (unsigned)(b - 4 * nf - 1), nb = (unsigned)(gridDim.x - 4 * nf - 1);
    mcc_candidates(st, threadIdx.x * nb + m, nb * blockDim.x);
  }
}

// Three blocks per diode, one per species: deterministic hole filling of the
// species' absorbed slots (the ordered list k_mid left in dead_buf), then
// its appends -- thermionic electrons (species 0), ionisation children
// sorted by parent id and replenished pairs (species 1 and 2) -- with ids and
// slots every block derives from counts it can read (events, emission
// count, ions absorbed).  The ion block also closes the diode's step (window
// tallies, next id, step counter) as soon as it has the counts; no block
// waits for another.
__global__ void __launch_bounds__(kPostThreads, 1) k_post(DevState st) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int ws32[32];
  __shared__ InstConst ic;
  __shared__ int sE, sNemit, sDi;

  const int inst = blockIdx.x / 3, sp = blockIdx.x - 3 * inst;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (blockIdx.x == 0 && tid == 0) {
    // k_mid has consumed the candidates
    if (*st.cand_count > (unsigned)st.cand_cap) atomicOr(&st.dyn[0].err, ERR_CAPACITY);
    *st.cand_count = 0u;
  }
  {
    const int* src = reinterpret_cast<const int*>(st.ic + inst);
    int* dst = reinterpret_cast<int*>(&ic);
    for (int w = tid; w < (int)(sizeof(InstConst) / 4); w += nt) dst[w] = src[w];
  }
  InstDyn* dyn = st.dyn + inst;
  PostScratch* ps = st.post + inst;
  const long long step = ps->step;
  const uint32_t base_id = ps->base_id;
  // every thread reads the counts itself (in the round trip of the constants)
  const int D = ps->D[sp], N = ps->N[sp];
  const int g = inst * 3 + sp;
  const long long off = st.seg_off[g];
  const int cap = st.seg_cap[g];
  if (tid == 0) {
    int e = dyn->ev_count;
    if (e > kEvCap) {
      atomicOr(&dyn->err, ERR_CAPACITY);
      e = kEvCap;
    }
    sE = e;
    sDi = ps->D[2];
  }
  // the ordered absorbed list, staged in shared memory when it fits
  uint32_t* dd = st.dead_buf + off;
  if (D <= kDeadSmem) {
    uint32_t* dd_s = reinterpret_cast<uint32_t*>(smem);
    for (int k = tid; k < D; k += nt) dd_s[k] = dd[k];
    dd = dd_s;
  }
  __syncthreads();                 // ic, the counts and the list are read by every thread below
  if (tid == 0) sNemit = emitted_count(ic, step);
  if (sp == 2 && tid == 0) {
    // ---- the diode's step closes here, while the blocks work on: window
    // tallies, ids, step.  Nothing in this kernel reads what this writes
    // (the step and first id come from PostScratch, the event count is
    // reset by the next push).
    const int Nem = sNemit, Ev = sE;
    const int Pt = ic.replenish ? ps->D[2] : 0;
    const uint32_t id_end = base_id + 2u * (uint32_t)Ev + (uint32_t)Nem + 2u * (uint32_t)Pt;
    dyn->next_id = id_end;
    // ids key the random streams: a diode that has handed out all 2^32 of
    // them would reuse one, so that is reported as running out of capacity
    if ((unsigned long long)base_id + 2ull * (unsigned)Ev + (unsigned)Nem + 2ull * (unsigned)Pt >
        0xFFFFFFFFull)
      atomicOr(&dyn->err, ERR_CAPACITY);
    if (step >= ic.window_start) {
      dyn->win_steps += 1;
      for (int k = 0; k < 3; ++k)
        for (int w = 0; w < 2; ++w) {
          long long c = 0;
          double e = 0.0;
          for (int r = 0; r < st.kp; ++r) {       // k_mid's list blocks, in order
            c += ps->cnt[k][r][w];
            e += ps->ke[k][r][w];
          }
          dyn->count[k][w] += c;
          dyn->ke[k][w] += e;
        }
      dyn->emitted += Nem;
      dyn->replenished += Pt;
    }
    dyn->pushed += (long long)ps->N[0] + ps->N[1] + ps->N[2];
    dyn->emit_dep = 0;
    dyn->step = step + 1;
  }
  if (sp == 2) {
    // every k_mid field block has read the push's charge: clear it for the
    // next push
    int64_t* acc = st.rho_acc + ic.node_off;
    for (int j = tid; j <= ic.Nz; j += nt) acc[j] = 0;
  }

  // ---- hole filling: the dead slots below the new count take the live
  // particles above it, in order.  The species-0 block draws its first
  // emitted electrons while the first round's loads are in flight.
  const int Nn = N - D;
  constexpr int kEmitRegs = 2;
  float ez[kEmitRegs], evx[kEmitRegs], evy[kEmitRegs], evz[kEmitRegs];
  bool have_emit = false;
  {
    int lo = 0, hi = D;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if ((int)dd[mid] < Nn) lo = mid + 1; else hi = mid;
    }
    const int h = lo;
    // kPer consecutive tail slots per thread: one search, one block scan and
    // one gather-then-scatter round trip for up to kPer * nt of them
    constexpr int kPer = 4;
    int run = 0;
    for (int base = 0; base < D; base += kPer * nt) {
      const int k0 = base + kPer * tid;
      const int t0 = Nn + k0;
      int a2 = h, b2 = D;                        // first listed slot >= t0
      while (a2 < b2) {
        const int mid = (a2 + b2) >> 1;
        if ((int)dd[mid] < t0) a2 = mid + 1; else b2 = mid;
      }
      unsigned lm = 0u;
      int cnt = 0;
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        if (k0 + u < D) {
          if (a2 < D && (int)dd[a2] == t0 + u) {
            ++a2;                                // absorbed: not moved
          } else {
            lm |= 1u << u;
            ++cnt;
          }
        }
      }
      int tot;
      int r = block_exclusive_scan<int>(cnt, &tot, ws32) + run;
      float z[kPer], vx[kPer], vy[kPer], vz[kPer];
      uint32_t id[kPer];
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        if (lm & (1u << u)) {
          const long long src = off + t0 + u;
          z[u] = st.z[src];
          vx[u] = st.vx[src];
          vy[u] = st.vy[src];
          vz[u] = st.vz[src];
          id[u] = st.id[src];
        }
      }
      if (sp == 0 && base == 0) {
        const int Ne = sNemit;                   // written before the scan's barriers
#pragma unroll
        for (int j = 0; j < kEmitRegs; ++j)
          if (tid + j * nt < Ne)
            emitted_electron(ic, tid + j * nt, step, ez[j], evx[j], evy[j], evz[j]);
        have_emit = true;
      }
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        if (lm & (1u << u)) put_particle(st, off, dd[r++], z[u], vx[u], vy[u], vz[u], id[u]);
      }
      run += tot;
    }
    __syncthreads();                 // shared memory is reused below
  }

  // ---- appends of this species (their charge is in the field already)
  const int E = sE, Nemit = sNemit;
  const int P = !ic.replenish ? 0 : (sp == 0 ? 0 : sDi);
  const uint32_t id_emit = base_id + 2u * (uint32_t)E;
  const uint32_t id_repl = id_emit + (uint32_t)Nemit;
  bool overflow = false;
  int newN = Nn;
  if (sp == 0) {
    int k = tid;
#pragma unroll
    for (int j = 0; j < kEmitRegs; ++j, k += nt) {
      if (k < Nemit) {
        float z = ez[j], vx = evx[j], vy = evy[j], vz = evz[j];
        if (!have_emit) emitted_electron(ic, k, step, z, vx, vy, vz);
        const long long sl = (long long)Nn + k;
        if (sl < cap) put_particle(st, off, sl, z, vx, vy, vz, id_emit + (uint32_t)k);
        else overflow = true;
      }
    }
    for (; k < Nemit; k += nt) {
      float z, vx, vy, vz;
      emitted_electron(ic, k, step, z, vx, vy, vz);
      const long long sl = (long long)Nn + k;
      if (sl < cap) put_particle(st, off, sl, z, vx, vy, vz, id_emit + (uint32_t)k);
      else overflow = true;
    }
    newN = min(Nn + Nemit, cap);
  } else {
    const uint32_t idb = (sp == 2) ? 1u : 0u;
    // ionisation children (Sec. 2.2 reading): the electron as a plasma
    // electron, the ion at the neutral's velocity, ordered by parent id
    unsigned long long* evk = reinterpret_cast<unsigned long long*>(smem);
    const Event* evb = st.ev_buf + (long long)inst * kEvCap;
    sort_events(evb, E, evk);
    for (int k = tid; k < E; k += nt) {
      const Event ev = evb[(int)(evk[k] & 0xffffffffu)];
      const long long sl = (long long)Nn + k;
      if (sl < cap) {
        const bool ion = sp == 2;
        put_particle(st, off, sl, ev.z, ion ? ev.vi[0] : ev.ve[0], ion ? ev.vi[1] : ev.ve[1],
                     ion ? ev.vi[2] : ev.ve[2], base_id + 2u * k + idb);
      } else {
        overflow = true;
      }
    }
    // replenishment (Sec. 2.1): one e-ion pair at a common uniform position
    // per ion absorbed; both blocks draw the pair's numbers
    const float sig = (sp == 2) ? ic.sig_i0 : ic.sig_e0;
    for (int k = tid; k < P; k += nt) {
      const uint4 A = philox10(make_uint4((uint32_t)k, (uint32_t)step, 0u, TAG_REPL), ic.key0[kStreamInject], ic.key1);
      const uint4 B = philox10(make_uint4((uint32_t)k, (uint32_t)step, 1u, TAG_REPL), ic.key0[kStreamInject], ic.key1);
      float gg[6];
      box_muller(A.x, A.y, gg[0], gg[1]);
      box_muller(A.z, A.w, gg[2], gg[3]);
      box_muller(B.x, B.y, gg[4], gg[5]);
      const float z = u01f(B.z) * ic.L_f;
      const long long sl = (long long)Nn + E + k;
      if (sl < cap) {
        const bool ion = sp == 2;
        put_particle(st, off, sl, z, sig * (ion ? gg[3] : gg[0]), sig * (ion ? gg[4] : gg[1]),
                     sig * (ion ? gg[5] : gg[2]), id_repl + 2u * k + idb);
      } else {
        overflow = true;
      }
    }
    newN = min(Nn + E + P, cap);
  }
  if (__syncthreads_or(overflow) && tid == 0) atomicOr(&dyn->err, ERR_CAPACITY);
  if (tid == 0) st.seg_count[g] = newN;
}

// ------------------------------------------------------------------ profiles
// Species density samples for the Sec. 3 late-time profiles: after a sampled
// step every particle of a species is binned with the charge's linear-weight
// rule (2^24 units per particle, no sign or weight) into a block histogram,
// which is added to the species' sums.  Grid (x, segment): the x blocks of a
// segment stride over its particles; the launch sizes x so that no block sees
// more than 2^20 particles (the 32-bit counters' bound).  Steps that are not
// samples return at once.
__global__ void __launch_bounds__(256) k_profile(DevState st) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int g = blockIdx.y;
  const int inst = g / 3, sp = g - 3 * inst;
  const InstConst& ic = st.ic[inst];
  if (!profile_due(st.prof_period, ic.window_start, st.dyn[inst].step - 1)) return;
  const int Nz = ic.Nz;
  const Hist h{reinterpret_cast<unsigned*>(smem)};
  hist_zero(h, Nz);
  __syncthreads();
  const int n = st.seg_count[g];
  const float* zs = st.z + st.seg_off[g];
  const float inv = ic.inv_dz_f;
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int i = base + threadIdx.x;
    float zz[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    unsigned am = 0u;
    if (i < n) {
      zz[0] = zs[i];
      am = 1u;
    }
    deposit_warp(h, zz, am, inv, Nz, true);
  }
  __syncthreads();
  hist_flush(h, Nz, 1LL, st.prof + (long long)sp * st.tn + ic.node_off);
}

// ------------------------------------------------------------------ helpers
__global__ void k_fill_ids(uint32_t* id, long long n, uint32_t first) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) id[i] = first + (uint32_t)i;
}

__global__ void k_count_outside(const float* z, long long n, float Lf, int* bad) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int b = 0;
  if (i < n) {
    const float v = z[i];
    b = !(v >= 0.0f && v < Lf);
  }
  if (__syncthreads_or(b) && threadIdx.x == 0) atomicAdd(bad, 1);
}

}  // namespace pic
