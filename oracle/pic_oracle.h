/*
 * pic_oracle.h -- CPU oracle of the 1D-3V electrostatic PIC-MCC thermionic
 * He diode (arXiv 2605.07083, Sec. 2.1-2.4, Eq. 1-8).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded FP64
 * restatement of the method, written to be checked by eye against the paper.
 * It shares no code, header, constant or helper with the CUDA library.  Only
 * tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg
 * may load it; the product path never does.
 *
 * Step order of one time step n -> n+1 (the paper does not spell out the
 * order; this is the reading used on both sides):
 *   1. rho^n from z^n with the 64-bit fixed-point linear-weighting rule
 *   2. Poisson, Dirichlet phi(0)=0, phi(L)=V (Sec. 2.1), Thomas algorithm
 *   3. E^n = -dphi/dz on nodes
 *   4. gather E(z^n) + leapfrog push (only v_z is accelerated, 1D-3V)
 *   5. wall absorption z<0 (cathode) / z>=L (anode) with count + KE tallies
 *   6. null-collision MCC on survivors (Sec. 2.2, Vahedi-Surendra scheme):
 *      candidate word from Philox2x32-10, collision draws from Philox4x32-10
 *   7. append ionisation children (by parent id), thermionic electrons
 *      (Sec. 2.2), replenished e-ion pairs (Sec. 2.1)
 *   8. remove absorbed particles
 *
 * Species: 0 = emitted electrons, 1 = plasma electrons, 2 = He+ ions.
 * Walls:   0 = cathode (z=0),     1 = anode (z=L).
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double L;            /* gap length, m */
    double V;            /* anode potential phi(L), V; phi(0) = 0 */
    int32_t Nz;          /* number of cells */
    int32_t replenish;   /* 1: re-inject one e-ion pair per absorbed ion (Sec. 2.1) */
    double dt;           /* time step, s */
    double gamma_emit;   /* imposed emitted flux, m^-2 s^-1 (Sec. 2.2) */
    double T_wall_K;     /* emission temperature T_c, K */
    double n_gas;        /* neutral He density, m^-3 */
    double T_gas_e_K;    /* neutral partner temperature for e-He, K */
    double T_gas_i_K;    /* neutral partner temperature for He+-He, K */
    double T_e0_eV;      /* replenished electron temperature, eV */
    double T_i0_eV;      /* replenished ion temperature, eV */
    double weight;       /* planar macro-particle weight, m^-2 */
    double m_ion;        /* He+ mass, kg */
    double m_gas;        /* He atom mass, kg */
    double sigma_el_e;   /* e-He elastic, m^2 (constant) */
    double sigma_cx_i;   /* He+-He charge exchange, m^2 (constant) */
    double sigma_el_i;   /* He+-He elastic, m^2 (constant) */
    double E_exc_eV;     /* excitation threshold, eV */
    double sigma_exc0;   /* excitation fit sigma0 (0 disables), m^2 */
    double E_iz_eV;      /* ionisation threshold P, eV */
    double lotz_a;       /* Lotz a (0 disables), m^2 eV^2 */
    double lotz_q;       /* Lotz q (shell electrons) */
    double E_cap_e_eV;   /* bound on e-He relative energy for nu_max, eV */
    double E_cap_i_eV;   /* bound on He+-He relative energy for nu_max, eV */
    int64_t window_start;/* first step counted in the averaging window */
    uint64_t seed;
} ocfg;

/* Window tallies.  count/ke indexed [species][wall]; ke in J m^-2. */
typedef struct {
    int64_t steps;              /* steps inside the window */
    int64_t count[3][2];
    double  ke[3][2];
    int64_t emitted;            /* thermionic macro-electrons emitted */
    int64_t replenished;        /* e-ion pairs re-injected */
    int64_t coll[6];            /* 0 null,1 e-el,2 exc,3 iz,4 cx,5 i-el */
    int64_t candidates[3];
    int64_t cap_exceeded;       /* candidates with nu_total > nu_max */
} otally;

/* Diagnostics of Sec. 2.3-2.4 (fluxes m^-2 s^-1, powers W m^-2). */
typedef struct {
    double window_time;
    double gamma_emit, gamma_emit_realized, gamma_ref, gamma_net, gamma_anode;
    double backflow_ratio, net_efficiency, collection_efficiency;
    double T_c_eV, W_F_eff, q_emit_theory;
    double q_back_em_cath, q_back_p_cath, q_ion_cath, gamma_ion_cath, q_ion_cath_recomb;
    double q_cooling_1, q_cooling_2;
    double q_out_em_anode, q_out_p_anode, q_ion_anode, gamma_ion_anode, q_ion_anode_recomb;
    double q_anode_total_1, q_anode_total_2;
} odiag;

/* One MCC candidate of the last step (for decision-margin checks). */
typedef struct {
    int32_t species;
    uint32_t id;
    int32_t process;     /* 0 null,1 e-el,2 exc,3 iz,4 cx,5 i-el */
    double margin;       /* min_k |U nu_max - cumulative nu_k| / nu_max */
} oevent;

typedef struct oracle_sim oracle_sim;

oracle_sim* oracle_create(const ocfg* cfg);
void    oracle_destroy(oracle_sim* s);
/* Append n particles (FP32 input, held as FP64); ids next_id, next_id+1, ... */
int     oracle_inject(oracle_sim* s, int species, int64_t n, const float* z,
                      const float* vx, const float* vy, const float* vz);
void    oracle_set_step(oracle_sim* s, int64_t step);
int64_t oracle_get_step(const oracle_sim* s);
uint32_t oracle_next_id(const oracle_sim* s);
void    oracle_step(oracle_sim* s, int64_t n_steps);
int64_t oracle_count(const oracle_sim* s, int species);
void    oracle_get_state(const oracle_sim* s, int species, double* z, double* vx,
                         double* vy, double* vz, uint32_t* id);
/* rho of the current state in fixed point (2^24 units of e*weight), Nz+1 */
void    oracle_rho_fixed(const oracle_sim* s, int64_t* out);
/* phi, E on the Nz+1 nodes from the current state */
void    oracle_field(const oracle_sim* s, double* phi, double* E);
void    oracle_tallies(const oracle_sim* s, otally* out);
void    oracle_diag(const oracle_sim* s, odiag* out);
int64_t oracle_events(const oracle_sim* s, oevent* out, int64_t cap);
/* derived constants: nu_max[3], candidate thresholds[3], emission x */
void    oracle_derived(const oracle_sim* s, double* nu_max, uint32_t* t_cand,
                       double* emit_x, uint32_t* t_frac);

/* Per-species linear-weight deposit of the current state, 2^24 units per
 * particle, no charge sign or weight (Nz+1 values). */
void    oracle_species_fixed(const oracle_sim* s, int species, int64_t* out);
/* Sampled profiles (Sec. 3 averaged potential; reading): after every step n
 * with n >= window_start and (n - window_start) % period == 0, phi of the
 * state after the step is added to phi_sum[Nz+1] and each species' deposit
 * to counts[3][Nz+1].  Setting the period (0 = off) clears the sums. */
void    oracle_set_profile_period(oracle_sim* s, int64_t period);
/* copies the sums (either pointer may be NULL); returns the sample count */
int64_t oracle_profiles(const oracle_sim* s, double* phi_sum, int64_t* counts);

/* ---- stand-alone pieces, exposed for pinning tests ---- */
void    oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* word 0 of Philox2x32-10 of counter (c0, c1) under key */
uint32_t oracle_philox2x32_10_w0(uint32_t c0, uint32_t c1, uint32_t key);
/* tridiag(-1,2,-1) phi = rhs on interior nodes 1..Nz-1, phi0 = 0, phiNz = V */
void    oracle_thomas(int32_t Nz, double V, const double* rhs, double* phi);
/* two-body isotropic-CM elastic scattering with |g'| = gnew */
void    oracle_two_body(double m, double M, const double v[3], const double vn[3],
                        double gnew, uint32_t r_cos, uint32_t r_phi,
                        double v_out[3], double vn_out[3]);
/* Eq. 1-8 from window tallies; counts as doubles so table values can be fed */
void    oracle_postprocess(double gamma_emit, double T_c_eV, double weight,
                           double window_time, const double count[3][2],
                           const double ke[3][2], double emitted, odiag* out);
double  oracle_sigma_exc(const ocfg* c, double E_eV);
double  oracle_sigma_iz(const ocfg* c, double E_eV);

#ifdef __cplusplus
}
#endif
#endif
