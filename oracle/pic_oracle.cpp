/*
 * pic_oracle.cpp -- plain FP64 single-threaded PIC-MCC oracle.
 *
 * TEST INFRASTRUCTURE ONLY (see pic_oracle.h).  Written from arXiv 2605.07083:
 *   Sec. 2.1  grid, Dirichlet Poisson every step, E = -grad(phi), absorbing
 *             electrodes, ion-loss replenishment with e-ion pairs
 *   Sec. 2.2  N_emit = Gamma*dt/w with stochastic fraction, half-Maxwellian
 *             emission at T_c, z_p = v_z dt, separate emitted/plasma electron
 *             populations, MCC (null collision, Vahedi & Surendra 1995) with
 *             constant e-He elastic and He+-He CX cross-sections, neutral
 *             partner drawn at T_n,e / T_n,i, optional excitation channel
 *   Sec. 2.3  Gamma_net = Gamma_emit - Gamma_ref, backflow ratio
 *   Sec. 2.4  Eq. 1-8 boundary energy diagnostics
 *   Sec. 3    late-time averaged potential profile (the input of Eq. 9-10)
 *             and per-species density profiles, sampled every `period` steps
 * Readings where the paper is silent are listed in the repository design
 * notes; each is marked "reading" below.
 *
 * Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared.  Contraction must
 * stay off: the fixed-point deposit rule is an exact FP32 operation sequence.
 */
#include "pic_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

/* CODATA 2018 */
const double kQe   = 1.602176634e-19;
const double kMe   = 9.1093837015e-31;
const double kEps0 = 8.8541878128e-12;
const double kKb   = 1.380649e-23;
const double kPi   = 3.14159265358979323846;
const double kEionHe = 24.59;          /* Sec. 2.4, first ionisation energy of He */
const double kTwo24 = 16777216.0;

enum { TAG_MCC = 1, TAG_EMIT = 2, TAG_EMIT_N = 3, TAG_REPL = 4 };
enum { STREAM_INJECT = 3 };

/* ---------------- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) -------
 * Each round: two 32x32->64 products of counter words 0 and 2 with the round
 * multipliers, the high halves mixed with the other counter words and the
 * round key, the words permuted; the key is bumped by the Weyl constants
 * between rounds. */
struct Ctr { uint32_t w[4]; };

Ctr philox10(Ctr c, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * c.w[0];
        uint64_t p1 = (uint64_t)M1 * c.w[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        Ctr n;
        n.w[0] = hi1 ^ c.w[1] ^ k0;
        n.w[1] = lo1;
        n.w[2] = hi0 ^ c.w[3] ^ k1;
        n.w[3] = lo0;
        c = n;
    }
    return c;
}

/* Philox2x32-10 (same paper): one 32x32->64 product per round on a 2-word
 * counter, key bumped by the Weyl constant.  Used for the per-particle
 * null-collision candidate word, drawn for every particle every step. */
uint32_t philox2x32_10_w0(uint32_t c0, uint32_t c1, uint32_t k) {
    const uint32_t M = 0xD256D193u, W = 0x9E3779B9u;
    for (int r = 0; r < 10; ++r) {
        if (r > 0) k += W;
        uint64_t p = (uint64_t)M * c0;
        uint32_t hi = (uint32_t)(p >> 32), lo = (uint32_t)p;
        c0 = hi ^ k ^ c1;
        c1 = lo;
    }
    return c0;
}

/* candidate key of a stream: seed_lo ^ stream*0x9E3779B9 ^ seed_hi */
uint32_t cand_key(uint64_t seed, uint32_t stream) {
    return (uint32_t)seed ^ (uint32_t)(stream * 0x9E3779B9u) ^ (uint32_t)(seed >> 32);
}

/* reading: key = (seed_lo ^ stream*0x9E3779B9, seed_hi); counter = (index,
 * step, draw block, tag).  stream = species for MCC, 3 for injection. */
Ctr draw(uint64_t seed, uint32_t stream, uint32_t index, int64_t step,
         uint32_t block, uint32_t tag) {
    uint32_t k0 = (uint32_t)seed ^ (uint32_t)(stream * 0x9E3779B9u);
    uint32_t k1 = (uint32_t)(seed >> 32);
    Ctr c = {{index, (uint32_t)step, block, tag}};
    return philox10(c, k0, k1);
}

/* open-interval uniform on the 2^-23 grid: (k + 1/2) 2^-23, k = r >> 9 */
double u01(uint32_t r) { return ((double)(r >> 9) + 0.5) * (1.0 / 8388608.0); }

/* Box-Muller: two standard normals from two uniforms */
void box_muller(uint32_t a, uint32_t b, double* n0, double* n1) {
    double rad = std::sqrt(-2.0 * std::log(u01(a)));
    double th = 2.0 * kPi * u01(b);
    *n0 = rad * std::cos(th);
    *n1 = rad * std::sin(th);
}

/* isotropic unit vector: cos(chi) = 1 - 2U, azimuth 2 pi U' */
void iso_dir(uint32_t rc, uint32_t rp, double d[3]) {
    double c = 1.0 - 2.0 * u01(rc);
    double s = std::sqrt(std::max(0.0, 1.0 - c * c));
    double ph = 2.0 * kPi * u01(rp);
    d[0] = s * std::cos(ph);
    d[1] = s * std::sin(ph);
    d[2] = c;
}

struct Species {
    std::vector<double> z, vx, vy, vz;
    std::vector<uint32_t> id;
    size_t size() const { return z.size(); }
    void push(double z_, double vx_, double vy_, double vz_, uint32_t id_) {
        z.push_back(z_); vx.push_back(vx_); vy.push_back(vy_); vz.push_back(vz_);
        id.push_back(id_);
    }
};

struct Child { uint32_t parent; double z; double ve[3]; double vi[3]; };

}  // namespace

struct oracle_sim {
    ocfg c;
    double dz;
    float inv_dz_f;
    double q[3], m[3], mu[3], gmax[3], nu_max[3];
    uint32_t t_cand[3];
    double emit_x;
    int64_t emit_floor;
    uint32_t t_frac;
    Species sp[3];
    uint32_t next_id;
    int64_t step;
    otally win;
    std::vector<oevent> events;
    /* sampled profiles (0 = off) */
    int64_t prof_period = 0;
    int64_t prof_n = 0;
    std::vector<double> phi_sum;     /* [Nz+1] */
    std::vector<int64_t> prof;       /* [3][Nz+1] */
};

/* ------------------------------------------------------------------------ */
extern "C" {

uint32_t oracle_philox2x32_10_w0(uint32_t c0, uint32_t c1, uint32_t key) {
    return philox2x32_10_w0(c0, c1, key);
}

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    Ctr c = {{ctr[0], ctr[1], ctr[2], ctr[3]}};
    Ctr r = philox10(c, key[0], key[1]);
    for (int i = 0; i < 4; ++i) out[i] = r.w[i];
}

/* Excitation: reading -- the paper's dataset is not available; fit
 * sigma0 (1 - E_th/E) above threshold. */
double oracle_sigma_exc(const ocfg* c, double E) {
    if (c->sigma_exc0 <= 0.0 || E <= c->E_exc_eV) return 0.0;
    return c->sigma_exc0 * (1.0 - c->E_exc_eV / E);
}

/* Ionisation: Lotz form a q ln(E/P) / (E P) above P (not in the paper). */
double oracle_sigma_iz(const ocfg* c, double E) {
    double P = c->E_iz_eV;
    if (c->lotz_a <= 0.0 || E <= P) return 0.0;
    return c->lotz_a * c->lotz_q * std::log(E / P) / (E * P);
}

/* Textbook Thomas algorithm for -phi_{j-1} + 2 phi_j - phi_{j+1} = rhs_j. */
void oracle_thomas(int32_t Nz, double V, const double* rhs, double* phi) {
    int n = Nz - 1;                    /* unknowns phi_1..phi_{Nz-1} */
    phi[0] = 0.0;
    phi[Nz] = V;
    if (n <= 0) return;
    std::vector<double> cp(n), dp(n);
    for (int i = 0; i < n; ++i) {
        double d = rhs[i + 1];
        if (i == 0) d += phi[0];
        if (i == n - 1) d += phi[Nz];
        double a = -1.0, b = 2.0, cc = -1.0;
        if (i == 0) {
            cp[i] = cc / b;
            dp[i] = d / b;
        } else {
            double den = b - a * cp[i - 1];
            cp[i] = cc / den;
            dp[i] = (d - a * dp[i - 1]) / den;
        }
    }
    phi[n] = dp[n - 1];
    for (int i = n - 2; i >= 0; --i) phi[i + 1] = dp[i] - cp[i] * phi[i + 2];
}

void oracle_two_body(double m, double M, const double v[3], const double vn[3],
                     double gnew, uint32_t r_cos, uint32_t r_phi,
                     double v_out[3], double vn_out[3]) {
    double d[3];
    iso_dir(r_cos, r_phi, d);
    for (int k = 0; k < 3; ++k) {
        double vcm = (m * v[k] + M * vn[k]) / (m + M);
        v_out[k] = vcm + M / (m + M) * gnew * d[k];
        vn_out[k] = vcm - m / (m + M) * gnew * d[k];
    }
}

/* Sec. 2.3 / Eq. 1-8. */
void oracle_postprocess(double gamma_emit, double T_c, double w, double T,
                        const double count[3][2], const double ke[3][2],
                        double emitted, odiag* o) {
    std::memset(o, 0, sizeof(*o));
    o->window_time = T;
    if (T <= 0.0) return;
    o->gamma_emit = gamma_emit;
    o->gamma_emit_realized = emitted * w / T;
    o->gamma_ref = count[0][0] * w / T;
    o->gamma_anode = count[0][1] * w / T;
    o->gamma_net = gamma_emit - o->gamma_ref;
    if (gamma_emit > 0.0) {
        o->backflow_ratio = o->gamma_ref / gamma_emit;
        o->net_efficiency = o->gamma_net / gamma_emit;
        o->collection_efficiency = o->gamma_anode / gamma_emit;
    }
    o->T_c_eV = T_c;
    /* Eq. 2 with A_R = 1.20e6 / (k_B/e)^2 in A m^-2 eV^-2 */
    double kb_over_e = kKb / kQe;
    double A_R = 1.20e6 / (kb_over_e * kb_over_e);
    if (gamma_emit > 0.0 && T_c > 0.0) {
        o->W_F_eff = -T_c * std::log(kQe * gamma_emit / (A_R * T_c * T_c));
        o->q_emit_theory = gamma_emit * kQe * (o->W_F_eff + 2.0 * T_c);   /* Eq. 1 */
    }
    o->q_back_em_cath = ke[0][0] / T;
    o->q_back_p_cath = ke[1][0] / T;
    o->q_ion_cath = ke[2][0] / T;
    o->gamma_ion_cath = count[2][0] * w / T;
    o->q_ion_cath_recomb = o->gamma_ion_cath * kQe * kEionHe;          /* Eq. 3 */
    o->q_cooling_1 = o->q_emit_theory - o->q_back_em_cath - o->q_back_p_cath
                     - o->q_ion_cath;                                  /* Eq. 4 */
    o->q_cooling_2 = o->q_cooling_1 - o->q_ion_cath_recomb;            /* Eq. 5 */
    o->q_out_em_anode = ke[0][1] / T;
    o->q_out_p_anode = ke[1][1] / T;
    o->q_ion_anode = ke[2][1] / T;
    o->q_anode_total_1 = o->q_out_em_anode + o->q_out_p_anode + o->q_ion_anode; /* Eq. 6 */
    o->gamma_ion_anode = count[2][1] * w / T;
    o->q_ion_anode_recomb = o->gamma_ion_anode * kQe * kEionHe;        /* Eq. 7 */
    o->q_anode_total_2 = o->q_anode_total_1 + o->q_ion_anode_recomb;   /* Eq. 8 */
}

oracle_sim* oracle_create(const ocfg* cfg) {
    if (!cfg || cfg->Nz < 1 || !(cfg->L > 0.0) || !(cfg->dt > 0.0) || !(cfg->weight > 0.0))
        return nullptr;
    oracle_sim* s = new oracle_sim();
    s->c = *cfg;
    const ocfg& c = s->c;
    s->dz = c.L / c.Nz;
    s->inv_dz_f = (float)((double)c.Nz / c.L);
    s->q[0] = s->q[1] = -kQe;
    s->q[2] = kQe;
    s->m[0] = s->m[1] = kMe;
    s->m[2] = c.m_ion;
    /* null-collision bound: nu_max = n * max_E(sum sigma) * g_max(E_cap) */
    double smax_e = c.sigma_el_e;
    if (c.sigma_exc0 > 0.0 && c.E_cap_e_eV > c.E_exc_eV)
        smax_e += c.sigma_exc0 * (1.0 - c.E_exc_eV / c.E_cap_e_eV);
    if (c.lotz_a > 0.0 && c.E_cap_e_eV > c.E_iz_eV) {
        double P = c.E_iz_eV, Epk = P * std::exp(1.0);
        if (c.E_cap_e_eV >= Epk) smax_e += c.lotz_a * c.lotz_q / (std::exp(1.0) * P * P);
        else smax_e += c.lotz_a * c.lotz_q * std::log(c.E_cap_e_eV / P) / (c.E_cap_e_eV * P);
    }
    double smax_i = c.sigma_cx_i + c.sigma_el_i;
    for (int k = 0; k < 3; ++k) {
        s->mu[k] = s->m[k] * c.m_gas / (s->m[k] + c.m_gas);
        double Ecap = (k < 2) ? c.E_cap_e_eV : c.E_cap_i_eV;
        s->gmax[k] = std::sqrt(2.0 * Ecap * kQe / s->mu[k]);
        double smax = (k < 2) ? smax_e : smax_i;
        s->nu_max[k] = c.n_gas * smax * s->gmax[k];
        double P = -std::expm1(-s->nu_max[k] * c.dt);
        s->t_cand[k] = (P >= 1.0) ? 0xFFFFFFFFu : (uint32_t)(P * 4294967296.0);
    }
    s->emit_x = (c.gamma_emit * c.dt) / c.weight;
    double fl = std::floor(s->emit_x);
    s->emit_floor = (int64_t)fl;
    s->t_frac = (uint32_t)((s->emit_x - fl) * 4294967296.0);
    s->next_id = 0;
    s->step = 0;
    std::memset(&s->win, 0, sizeof(s->win));
    return s;
}

void oracle_destroy(oracle_sim* s) { delete s; }

int oracle_inject(oracle_sim* s, int sp, int64_t n, const float* z, const float* vx,
                  const float* vy, const float* vz) {
    if (sp < 0 || sp > 2 || n < 0) return -1;
    for (int64_t i = 0; i < n; ++i)
        s->sp[sp].push(z[i], vx[i], vy[i], vz[i], s->next_id++);
    return 0;
}

void oracle_set_step(oracle_sim* s, int64_t step) { s->step = step; }
int64_t oracle_get_step(const oracle_sim* s) { return s->step; }
uint32_t oracle_next_id(const oracle_sim* s) { return s->next_id; }
int64_t oracle_count(const oracle_sim* s, int sp) { return (int64_t)s->sp[sp].size(); }

void oracle_get_state(const oracle_sim* s, int sp, double* z, double* vx, double* vy,
                      double* vz, uint32_t* id) {
    const Species& p = s->sp[sp];
    for (size_t i = 0; i < p.size(); ++i) {
        if (z) z[i] = p.z[i];
        if (vx) vx[i] = p.vx[i];
        if (vy) vy[i] = p.vy[i];
        if (vz) vz[i] = p.vz[i];
        if (id) id[i] = p.id[i];
    }
}

void oracle_derived(const oracle_sim* s, double* nu_max, uint32_t* t_cand, double* emit_x,
                    uint32_t* t_frac) {
    for (int k = 0; k < 3; ++k) {
        if (nu_max) nu_max[k] = s->nu_max[k];
        if (t_cand) t_cand[k] = s->t_cand[k];
    }
    if (emit_x) *emit_x = s->emit_x;
    if (t_frac) *t_frac = s->t_frac;
}

}  // extern "C"

namespace {

/* Fixed-point cell rule (reading): all in FP32, round to nearest:
 *   s = z * inv_dz, j = floor(s) clamped to [0, Nz-1], f = s - j (exact),
 *   Q = trunc(f * 2^24);  node j gets 2^24 - Q units, node j+1 gets Q. */
struct CellW { int j; float f; int64_t Q; };

CellW cell_of(float zf, float inv_dz, int Nz) {
    volatile float sv = zf * inv_dz;
    float s = sv;
    int j = (int)std::floor(s);
    if (j < 0) j = 0;
    if (j > Nz - 1) j = Nz - 1;
    volatile float fv = s - (float)j;
    float f = fv;
    volatile float qf = f * 16777216.0f;
    CellW r;
    r.j = j;
    r.f = f;
    r.Q = (int64_t)(float)qf;
    return r;
}

void deposit(const oracle_sim* s, std::vector<int64_t>& rho) {
    const int Nz = s->c.Nz;
    rho.assign(Nz + 1, 0);
    for (int k = 0; k < 3; ++k) {
        const int64_t sign = (k == 2) ? 1 : -1;
        const Species& p = s->sp[k];
        for (size_t i = 0; i < p.size(); ++i) {
            CellW cw = cell_of((float)p.z[i], s->inv_dz_f, Nz);
            rho[cw.j] += sign * ((int64_t)(1 << 24) - cw.Q);
            rho[cw.j + 1] += sign * cw.Q;
        }
    }
}

/* Linear-weight deposit of one species without charge sign or weight:
 * every particle puts 2^24 units on its two nodes (same cell rule). */
void deposit_species(const oracle_sim* s, int k, int64_t* out) {
    const int Nz = s->c.Nz;
    for (int j = 0; j <= Nz; ++j) out[j] = 0;
    const Species& p = s->sp[k];
    for (size_t i = 0; i < p.size(); ++i) {
        CellW cw = cell_of((float)p.z[i], s->inv_dz_f, Nz);
        out[cw.j] += (int64_t)(1 << 24) - cw.Q;
        out[cw.j + 1] += cw.Q;
    }
}

/* Sec. 2.1: phi from rho each step, E = -dphi/dz (central inside, one-sided
 * at the electrodes -- reading). */
void field(const oracle_sim* s, const std::vector<int64_t>& rho, std::vector<double>& phi,
           std::vector<double>& E) {
    const int Nz = s->c.Nz;
    const double dz = s->dz;
    /* rho_j [C m^-3] = rho_fix * e * w / (2^24 dz); rhs = dz^2 rho / eps0 */
    std::vector<double> rhs(Nz + 1, 0.0);
    for (int j = 1; j < Nz; ++j) {
        double rho_si = (double)rho[j] * kQe * s->c.weight / (kTwo24 * dz);
        rhs[j] = dz * dz * rho_si / kEps0;
    }
    phi.assign(Nz + 1, 0.0);
    oracle_thomas(Nz, s->c.V, rhs.data(), phi.data());
    E.assign(Nz + 1, 0.0);
    E[0] = -(phi[1] - phi[0]) / dz;
    E[Nz] = -(phi[Nz] - phi[Nz - 1]) / dz;
    for (int j = 1; j < Nz; ++j) E[j] = -(phi[j + 1] - phi[j - 1]) / (2.0 * dz);
}

double ke_of(double m, double vx, double vy, double vz, double w) {
    return 0.5 * m * (vx * vx + vy * vy + vz * vz) * w;
}

void do_step(oracle_sim* s) {
    const ocfg& c = s->c;
    const int Nz = c.Nz;
    const int64_t n = s->step;
    const bool in_win = n >= c.window_start;
    std::vector<int64_t> rho;
    std::vector<double> phi, E;
    deposit(s, rho);                                   /* 1 */
    field(s, rho, phi, E);                             /* 2, 3 */
    s->events.clear();
    std::vector<Child> children;
    int64_t ions_lost = 0;
    const double M = c.m_gas;

    for (int k = 0; k < 3; ++k) {
        Species& p = s->sp[k];
        const double qm_dt = s->q[k] / s->m[k] * c.dt;
        const double Tn = (k < 2) ? c.T_gas_e_K : c.T_gas_i_K;
        const double sig_n = std::sqrt(kKb * Tn / M);
        std::vector<char> alive(p.size(), 1);
        for (size_t i = 0; i < p.size(); ++i) {
            /* 4: gather with the deposit's linear weights, leapfrog */
            CellW cw = cell_of((float)p.z[i], s->inv_dz_f, Nz);
            double f = (double)cw.f;
            double Ez = (1.0 - f) * E[cw.j] + f * E[cw.j + 1];
            p.vz[i] += qm_dt * Ez;
            p.z[i] += p.vz[i] * c.dt;
            /* 5: absorbing electrodes (reading: z < 0 cathode, z >= L anode) */
            int wall = -1;
            if (p.z[i] < 0.0) wall = 0;
            else if (p.z[i] >= c.L) wall = 1;
            if (wall >= 0) {
                alive[i] = 0;
                if (k == 2) ++ions_lost;
                if (in_win) {
                    s->win.count[k][wall] += 1;
                    s->win.ke[k][wall] += ke_of(s->m[k], p.vx[i], p.vy[i], p.vz[i], c.weight);
                }
                continue;
            }
            /* 6: null-collision candidate test: Philox2x32 word 0 of
             * (id, step) under the species' candidate key */
            if (c.n_gas <= 0.0) continue;
            uint32_t rc = philox2x32_10_w0(p.id[i], (uint32_t)n, cand_key(c.seed, (uint32_t)k));
            if (!(rc < s->t_cand[k])) continue;
            Ctr A = draw(c.seed, (uint32_t)k, p.id[i], n, 0, TAG_MCC);
            if (in_win) s->win.candidates[k] += 1;
            Ctr B = draw(c.seed, (uint32_t)k, p.id[i], n, 1, TAG_MCC);
            double nn[4];
            box_muller(B.w[0], B.w[1], &nn[0], &nn[1]);
            box_muller(B.w[2], B.w[3], &nn[2], &nn[3]);
            double vn[3] = {sig_n * nn[0], sig_n * nn[1], sig_n * nn[2]};
            double v[3] = {p.vx[i], p.vy[i], p.vz[i]};
            double g[3] = {v[0] - vn[0], v[1] - vn[1], v[2] - vn[2]};
            double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
            double gm = std::sqrt(g2);
            double Erel = 0.5 * s->mu[k] * g2 / kQe;
            double x = u01(A.w[1]) * s->nu_max[k];
            double cum[3];
            int nproc;
            if (k < 2) {
                cum[0] = c.n_gas * c.sigma_el_e * gm;
                cum[1] = cum[0] + c.n_gas * oracle_sigma_exc(&c, Erel) * gm;
                cum[2] = cum[1] + c.n_gas * oracle_sigma_iz(&c, Erel) * gm;
                nproc = 3;
            } else {
                cum[0] = c.n_gas * c.sigma_cx_i * gm;
                cum[1] = cum[0] + c.n_gas * c.sigma_el_i * gm;
                nproc = 2;
            }
            if (cum[nproc - 1] > s->nu_max[k] && in_win) s->win.cap_exceeded += 1;
            int sel = nproc;                       /* nproc == null */
            for (int q = 0; q < nproc; ++q)
                if (x < cum[q]) { sel = q; break; }
            double margin = 1e300;
            for (int q = 0; q < nproc; ++q)
                margin = std::min(margin, std::fabs(x - cum[q]) / s->nu_max[k]);
            int code;
            double vo[3], vno[3];
            if (k < 2) {
                code = (sel == 0) ? 1 : (sel == 1) ? 2 : (sel == 2) ? 3 : 0;
                if (code == 1) {                              /* elastic, |g| kept */
                    oracle_two_body(s->m[k], M, v, vn, gm, A.w[2], A.w[3], vo, vno);
                    p.vx[i] = vo[0]; p.vy[i] = vo[1]; p.vz[i] = vo[2];
                } else if (code == 2) {                       /* excitation */
                    double gnew = std::sqrt(2.0 * (Erel - c.E_exc_eV) * kQe / s->mu[k]);
                    oracle_two_body(s->m[k], M, v, vn, gnew, A.w[2], A.w[3], vo, vno);
                    p.vx[i] = vo[0]; p.vy[i] = vo[1]; p.vz[i] = vo[2];
                } else if (code == 3) {                       /* ionisation */
                    Ctr C = draw(c.seed, (uint32_t)k, p.id[i], n, 2, TAG_MCC);
                    double Eex = Erel - c.E_iz_eV;
                    double U = u01(C.w[0]);
                    double E1 = U * Eex, E2 = (1.0 - U) * Eex;
                    double d1[3], d2[3];
                    iso_dir(A.w[2], A.w[3], d1);
                    iso_dir(C.w[1], C.w[2], d2);
                    double s1 = std::sqrt(2.0 * E1 * kQe / kMe);
                    double s2 = std::sqrt(2.0 * E2 * kQe / kMe);
                    p.vx[i] = vn[0] + s1 * d1[0];
                    p.vy[i] = vn[1] + s1 * d1[1];
                    p.vz[i] = vn[2] + s1 * d1[2];
                    Child ch;
                    ch.parent = p.id[i];
                    ch.z = p.z[i];
                    for (int d = 0; d < 3; ++d) {
                        ch.ve[d] = vn[d] + s2 * d2[d];
                        ch.vi[d] = vn[d];
                    }
                    children.push_back(ch);
                }
            } else {
                code = (sel == 0) ? 4 : (sel == 1) ? 5 : 0;
                if (code == 4) {                              /* CX: ion takes v_n */
                    p.vx[i] = vn[0]; p.vy[i] = vn[1]; p.vz[i] = vn[2];
                } else if (code == 5) {
                    oracle_two_body(s->m[k], M, v, vn, gm, A.w[2], A.w[3], vo, vno);
                    p.vx[i] = vo[0]; p.vy[i] = vo[1]; p.vz[i] = vo[2];
                }
            }
            if (in_win) s->win.coll[code] += 1;
            oevent ev;
            ev.species = k;
            ev.id = p.id[i];
            ev.process = code;
            ev.margin = margin;
            s->events.push_back(ev);
        }
        /* 8: remove absorbed (done here; appends below go to the tail) */
        Species keep;
        for (size_t i = 0; i < p.size(); ++i)
            if (alive[i]) keep.push(p.z[i], p.vx[i], p.vy[i], p.vz[i], p.id[i]);
        p = keep;
    }

    /* 7a: ionisation children, ordered by parent id; e then ion ids */
    std::sort(children.begin(), children.end(),
              [](const Child& a, const Child& b) { return a.parent < b.parent; });
    for (const Child& ch : children) {
        s->sp[1].push(ch.z, ch.ve[0], ch.ve[1], ch.ve[2], s->next_id++);
        s->sp[2].push(ch.z, ch.vi[0], ch.vi[1], ch.vi[2], s->next_id++);
    }
    /* 7b: thermionic emission (Sec. 2.2) */
    {
        int64_t N = s->emit_floor;
        if (s->t_frac > 0) {
            Ctr R = draw(c.seed, STREAM_INJECT, 0, n, 0, TAG_EMIT_N);
            if (R.w[0] < s->t_frac) N += 1;
        }
        const double sw = std::sqrt(kKb * c.T_wall_K / kMe);
        for (int64_t k = 0; k < N; ++k) {
            Ctr R = draw(c.seed, STREAM_INJECT, (uint32_t)k, n, 0, TAG_EMIT);
            double n0, n1;
            box_muller(R.w[0], R.w[1], &n0, &n1);
            /* reading: flux-weighted half-Maxwellian, v_z Rayleigh(sw) */
            double vz = sw * std::sqrt(-2.0 * std::log(u01(R.w[2])));
            s->sp[0].push(vz * c.dt, sw * n0, sw * n1, vz, s->next_id++);
        }
        if (in_win) s->win.emitted += N;
    }
    /* 7c: replenishment of e-ion pairs (Sec. 2.1) */
    if (c.replenish) {
        const double se = std::sqrt(c.T_e0_eV * kQe / kMe);
        const double si = std::sqrt(c.T_i0_eV * kQe / c.m_ion);
        for (int64_t k = 0; k < ions_lost; ++k) {
            Ctr A = draw(c.seed, STREAM_INJECT, (uint32_t)k, n, 0, TAG_REPL);
            Ctr B = draw(c.seed, STREAM_INJECT, (uint32_t)k, n, 1, TAG_REPL);
            double g[6];
            box_muller(A.w[0], A.w[1], &g[0], &g[1]);
            box_muller(A.w[2], A.w[3], &g[2], &g[3]);
            box_muller(B.w[0], B.w[1], &g[4], &g[5]);
            double z = u01(B.w[2]) * c.L;
            s->sp[1].push(z, se * g[0], se * g[1], se * g[2], s->next_id++);
            s->sp[2].push(z, si * g[3], si * g[4], si * g[5], s->next_id++);
        }
        if (in_win) s->win.replenished += ions_lost;
    }
    if (in_win) s->win.steps += 1;
    s->step = n + 1;
    /* profile sample of the state after step n (reading: the steps n >=
     * window_start with (n - window_start) a multiple of the period) */
    if (s->prof_period > 0 && n >= c.window_start && (n - c.window_start) % s->prof_period == 0) {
        std::vector<int64_t> rho;
        std::vector<double> ph, e;
        deposit(s, rho);
        field(s, rho, ph, e);
        for (int j = 0; j <= Nz; ++j) s->phi_sum[j] += ph[j];
        std::vector<int64_t> cnt(Nz + 1);
        for (int k = 0; k < 3; ++k) {
            deposit_species(s, k, cnt.data());
            for (int j = 0; j <= Nz; ++j) s->prof[(size_t)k * (Nz + 1) + j] += cnt[j];
        }
        s->prof_n += 1;
    }
}

}  // namespace

extern "C" {

void oracle_step(oracle_sim* s, int64_t n_steps) {
    for (int64_t i = 0; i < n_steps; ++i) do_step(s);
}

void oracle_rho_fixed(const oracle_sim* s, int64_t* out) {
    std::vector<int64_t> rho;
    deposit(s, rho);
    std::memcpy(out, rho.data(), rho.size() * sizeof(int64_t));
}

void oracle_field(const oracle_sim* s, double* phi, double* E) {
    std::vector<int64_t> rho;
    std::vector<double> ph, e;
    deposit(s, rho);
    field(s, rho, ph, e);
    if (phi) std::memcpy(phi, ph.data(), ph.size() * sizeof(double));
    if (E) std::memcpy(E, e.data(), e.size() * sizeof(double));
}

void oracle_tallies(const oracle_sim* s, otally* out) { *out = s->win; }

void oracle_diag(const oracle_sim* s, odiag* out) {
    double cnt[3][2], ke[3][2];
    for (int k = 0; k < 3; ++k)
        for (int w = 0; w < 2; ++w) {
            cnt[k][w] = (double)s->win.count[k][w];
            ke[k][w] = s->win.ke[k][w];
        }
    double T = (double)s->win.steps * s->c.dt;
    double Tc = kKb * s->c.T_wall_K / kQe;
    oracle_postprocess(s->c.gamma_emit, Tc, s->c.weight, T, cnt, ke, (double)s->win.emitted, out);
}

void oracle_species_fixed(const oracle_sim* s, int species, int64_t* out) {
    if (species < 0 || species > 2) return;
    deposit_species(s, species, out);
}

void oracle_set_profile_period(oracle_sim* s, int64_t period) {
    const int Nz = s->c.Nz;
    s->prof_period = period > 0 ? period : 0;
    s->prof_n = 0;
    s->phi_sum.assign(Nz + 1, 0.0);
    s->prof.assign((size_t)3 * (Nz + 1), 0);
}

int64_t oracle_profiles(const oracle_sim* s, double* phi_sum, int64_t* counts) {
    if (phi_sum && !s->phi_sum.empty())
        std::memcpy(phi_sum, s->phi_sum.data(), s->phi_sum.size() * sizeof(double));
    if (counts && !s->prof.empty())
        std::memcpy(counts, s->prof.data(), s->prof.size() * sizeof(int64_t));
    return s->prof_n;
}

int64_t oracle_events(const oracle_sim* s, oevent* out, int64_t cap) {
    int64_t n = (int64_t)s->events.size();
    for (int64_t i = 0; i < n && i < cap; ++i) out[i] = s->events[i];
    return n;
}

}  // extern "C"
