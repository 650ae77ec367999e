/*
 * pic.h -- C ABI of the GB300 PIC-MCC thermionic-diode library.
 *
 * The library advances 1D-in-space, 3D-in-velocity electrostatic
 * particle-in-cell / Monte Carlo collision models of planar He diodes with a
 * thermionically emitting cathode (arXiv 2605.07083, Sec. 2.1-2.4), one or
 * many independent diodes ("instances") per handle, on one CUDA device.
 *
 * Conventions for every entry point
 *   - Plain pointers and sizes only.  Pointers named "host" or used with
 *     on_device == 0 are host memory; with on_device != 0 they are device
 *     memory of the handle's device.  The caller owns every buffer it passes;
 *     the library reads or writes it only during the call (device buffers:
 *     until the call's work on the handle's stream has finished).
 *   - The library owns all simulation state (particles, grids, tallies).
 *   - Every function returns PIC_OK (0) or a negative PIC_E* code; nothing
 *     aborts or exits.  Work is enqueued on the handle's CUDA stream.
 *     Device-side failures (capacity overflow, null-collision bound exceeded)
 *     raise sticky flags that the next synchronising call returns.
 *   - Species: 0 = emitted (thermionic) electrons, 1 = plasma electrons,
 *     2 = He+ ions (Sec. 2.2 tracks emitted and plasma electrons separately).
 *     Walls: 0 = cathode at z = 0, 1 = anode at z = L.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_ABI_VERSION 1

enum {
    PIC_OK = 0,
    PIC_EINVAL = -1,      /* bad argument or configuration */
    PIC_ENOMEM = -2,      /* device allocation failed */
    PIC_ECUDA = -3,       /* a CUDA runtime call failed */
    PIC_ECAPACITY = -4,   /* a species outgrew its capacity (extra particles dropped), or a
                             diode used up its 2^32 particle ids (ids key the random
                             streams, so they are not reused) */
    PIC_ETIMEOUT = -5,    /* a bounded device wait gave up */
    PIC_EENERGYCAP = -6   /* a collision candidate exceeded the null-collision bound */
};

enum { PIC_SPECIES_EMITTED = 0, PIC_SPECIES_PLASMA_E = 1, PIC_SPECIES_ION = 2 };

/*
 * One diode.  Copied at pic_create.  Paper references:
 *   gap_m, bias_V, n_cells, dt_s: Sec. 2.1 (Dirichlet phi(0)=0, phi(L)=bias_V)
 *   gamma_emit, T_wall_K: Sec. 2.2 (imposed flux, emission temperature T_c)
 *   n_gas, sigma_el_e, sigma_cx_i, T_gas_e_K, T_gas_i_K: Sec. 2.2 (MCC)
 *   weight: Sec. 2.1 (planar macro-particle weight w0, m^-2; one value for
 *           all species of the instance)
 *   replenish, T_e0_eV, T_i0_eV: Sec. 2.1 (ion-loss replenishment)
 *   E_exc_eV, sigma_exc0: excitation channel, fit sigma0 (1 - E_th/E)
 *           (the paper's dataset is not published; sigma_exc0 = 0 disables)
 *   E_iz_eV, lotz_a, lotz_q: Lotz ionisation a q ln(E/P)/(E P) (not in the
 *           paper; lotz_a = 0 disables)
 *   E_cap_e_eV, E_cap_i_eV: bound on the relative collision energy used for
 *           the null-collision frequency nu_max (exceeding it raises
 *           PIC_EENERGYCAP)
 *   window_start: first step whose boundary fluxes enter the late-time
 *           averages of pic_diagnostics (Sec. 2.3)
 *   capacity: particle capacity per species (0 = choose automatically)
 */
typedef struct pic_config {
    uint32_t size;            /* sizeof(pic_config): ABI check */
    int32_t n_cells;          /* Nz, 1 <= Nz <= 4096 */
    double gap_m;             /* L, m */
    double bias_V;            /* phi(L), V */
    double dt_s;              /* time step, s */
    double gamma_emit;        /* m^-2 s^-1 */
    double T_wall_K;          /* emission temperature, K */
    double n_gas;             /* m^-3 */
    double T_gas_e_K;         /* neutral partner temperature for e-He, K */
    double T_gas_i_K;         /* neutral partner temperature for He+-He, K */
    double T_e0_eV;           /* replenished electron temperature, eV */
    double T_i0_eV;           /* replenished ion temperature, eV */
    double weight;            /* m^-2 */
    double m_ion;             /* kg */
    double m_gas;             /* kg */
    double sigma_el_e;        /* m^2 */
    double sigma_cx_i;        /* m^2 */
    double sigma_el_i;        /* m^2 */
    double E_exc_eV;
    double sigma_exc0;        /* m^2 */
    double E_iz_eV;
    double lotz_a;            /* m^2 eV^2 */
    double lotz_q;
    double E_cap_e_eV;
    double E_cap_i_eV;
    int32_t replenish;        /* 0 / 1 */
    int32_t reserved0;
    int64_t window_start;
    uint64_t seed;            /* Philox key material */
    int64_t capacity[3];
} pic_config;

/* Optional device allocator (e.g. a framework's caching allocator).  NULL in
 * pic_create means cudaMallocAsync / cudaFreeAsync on the handle's stream. */
typedef struct pic_allocator {
    void* (*alloc)(size_t bytes, void* cuda_stream, void* ctx);
    void (*free)(void* ptr, size_t bytes, void* cuda_stream, void* ctx);
    void* ctx;
} pic_allocator;

/* Launch shape and scheduling knobs (pic_tune).  Zero keeps the current value. */
typedef struct pic_tuning {
    uint32_t size;            /* sizeof(pic_tuning) */
    int32_t push_threads;     /* threads per block of the particle kernels (64..384, multiple of
                                 32; default: the size that keeps closest to 24 resident warps
                                 per SM for the handle's cell count, the first of 384, 256,
                                 128, 160, ... that does) */
    int32_t push_blocks_per_sm;  /* cap on resident blocks per SM (default: occupancy limit) */
    int32_t sort_period;      /* counting sort by cell every this many steps; < 0 disables */
    int32_t graph_steps;      /* longest step loop captured as one CUDA graph (default 64,
                                 at most 4096); every power of two below it is captured too,
                                 so pic_step(n) runs any n as graphs.  With a periodic sort
                                 the longest graph is rounded up to a multiple of the sort
                                 period, the shorter ones are the period times powers of two,
                                 and graphs start on sort-aligned steps only: pic_step runs
                                 single steps up to the next aligned step and for a remainder
                                 shorter than one period (no graphs at all when the period
                                 exceeds 4096).  Each is captured the first time a pic_step
                                 needs it (again after a change of launch shape).  < 0
                                 disables graphs */
    int32_t wait_polls;       /* polls of a bulk-copy wait in the push kernel before it gives
                                 up with PIC_ETIMEOUT (default 2^20, each suspending the warp
                                 up to ~1 us): n > 0 sets n; -1 gives up without polling, a
                                 way to exercise the time-out path (the kernel first lets its
                                 copies in flight land, so nothing faults); -2 restores the
                                 default */
    int32_t push_chunk;       /* quads each warp of the push streams per chunk, 32 or 64
                                 (default: 64 unless the cell grid's shared memory then
                                 leaves fewer resident warps per SM than 32 does) */
    int32_t reserved[1];
} pic_tuning;

/* Late-time diagnostics of one instance (Sec. 2.3, Eq. 1-8).  Fluxes in
 * m^-2 s^-1, energies in J m^-2, powers in W m^-2, temperatures in eV. */
typedef struct pic_diag {
    int64_t step;                 /* index of the next step to run */
    int64_t window_steps;         /* steps accumulated in the window */
    double window_time;           /* window_steps * dt */
    int64_t n_live[3];
    int64_t count[3][2];          /* absorbed macro-particles per species, wall */
    double ke[3][2];              /* absorbed kinetic energy * weight */
    int64_t emitted;              /* thermionic macro-electrons emitted */
    int64_t replenished;          /* e-ion pairs re-injected */
    int64_t collisions[6];        /* null, e-He elastic, excitation, ionisation, CX, He+-He elastic */
    int64_t candidates[3];        /* null-collision candidates per species */
    int64_t energy_cap_exceeded;
    int64_t particles_pushed;     /* particle-steps done since creation (all windows) */
    double gamma_emit, gamma_emit_realized, gamma_ref, gamma_net, gamma_anode;
    double backflow_ratio;        /* Gamma_ref / Gamma_emit */
    double net_efficiency;        /* Gamma_net / Gamma_emit */
    double collection_efficiency; /* Gamma_anode / Gamma_emit */
    double T_c_eV, W_F_eff, q_emit_theory;                               /* Eq. 1-2 */
    double q_back_em_cath, q_back_p_cath, q_ion_cath, gamma_ion_cath;
    double q_ion_cath_recomb;                                            /* Eq. 3 */
    double q_cooling_1, q_cooling_2;                                     /* Eq. 4-5 */
    double q_out_em_anode, q_out_p_anode, q_ion_anode, gamma_ion_anode;
    double q_anode_total_1, q_ion_anode_recomb, q_anode_total_2;         /* Eq. 6-8 */
    int32_t error_flags;          /* bit (-code - 1) set for each sticky PIC_E* code */
    int32_t reserved;
} pic_diag;

/* Per-kernel device time of pic_profile_steps, milliseconds (CUDA events). */
typedef struct pic_profile {
    int64_t steps;
    double ms_push;               /* gather+push+absorb+candidate test+deposit kernel */
    double ms_mcc;                /* collisions of the candidates, field solve of the new
                                     state and ordered absorbed lists (one kernel) */
    double ms_post;               /* compaction+injection kernel */
    double ms_sort;               /* counting sort kernels */
    double ms_total;
    int64_t particle_steps;       /* live particles pushed, summed over steps */
    int64_t launches;             /* kernels launched */
    int64_t push_launches;
} pic_profile;

typedef struct pic_handle pic_handle;

/* Create n_instances independent diodes on the current CUDA device.
 * cfgs: n_instances configs (host).  cuda_stream: cudaStream_t or NULL for
 * the legacy default stream.  alloc: optional device allocator.  The handle
 * starts empty at step 0.  Sec. 2.1 (grid, Poisson), 2.2 (MCC constants). */
int pic_create(const pic_config* cfgs, int n_instances, void* cuda_stream,
               const pic_allocator* alloc, pic_handle** out);

/* Append n particles of one species to an instance (Sec. 2.1 initial
 * loading).  z in [0, gap_m); velocities in m s^-1, FP32.  Particles get the
 * instance's next ids in order.  Returns PIC_ECAPACITY (nothing appended) if
 * they do not fit, PIC_EINVAL (nothing appended) if a z lies outside [0, L)
 * -- checked on the device after the copy, for host and device pointers
 * alike.  Synchronises the stream. */
int pic_inject(pic_handle* h, int instance, int species, int64_t n, const float* z,
               const float* vx, const float* vy, const float* vz, int on_device);

/* Advance every instance by n_steps time steps (Sec. 2.1-2.2 step: deposit,
 * Poisson, gather, push, absorb, MCC, emit, replenish, compact).
 * Asynchronous; returns a sticky error seen earlier, else PIC_OK. */
int pic_step(pic_handle* h, int64_t n_steps);

/* Capture now, from the current step, the CUDA graphs that pic_step(n_steps)
 * would launch, so that the call itself only launches (the first pic_step
 * that needs a graph otherwise captures it, a one-time host cost of about a
 * millisecond per 64 steps).  Runs no step; the charge and field of an
 * injected or loaded state are computed first, as pic_step would.  Returns a
 * sticky error seen earlier, PIC_EINVAL for a null handle or n_steps < 0, or
 * PIC_ECUDA if a capture fails. */
int pic_prepare_steps(pic_handle* h, int64_t n_steps);

/* Same steps as pic_step, launched one by one with CUDA events around each
 * kernel; synchronises and reports per-kernel device time (each kernel's
 * time includes its launch latency, which graphs hide in pic_step). */
int pic_profile_steps(pic_handle* h, int64_t n_steps, pic_profile* out);

/* Window tallies and Eq. 1-8 diagnostics of one instance.  Synchronises. */
int pic_diagnostics(pic_handle* h, int instance, pic_diag* out);

/* Copy out the live particles of one species.  cap = room in the buffers;
 * *n receives the live count (PIC_ECAPACITY if cap < *n, nothing copied).
 * Any buffer may be NULL.  Synchronises. */
int pic_get_state(pic_handle* h, int instance, int species, float* z, float* vx, float* vy,
                  float* vz, uint32_t* id, int64_t cap, int64_t* n, int on_device);

/* Fixed-point charge rho of the current state on the n_cells+1 nodes, in
 * units of e*weight/2^24 (signed).  Synchronises. */
int pic_get_rho_fixed(pic_handle* h, int instance, int64_t* out, int64_t n_nodes);

/* phi (V, FP64) and E (V/m, the FP32 copy the push gathers) on the nodes
 * for the current state; either pointer may be NULL.  A time step solves E
 * only; this call solves phi (and E, identically) from the current charge on
 * the handle's stream.  Synchronises. */
int pic_get_field(pic_handle* h, int instance, double* phi, float* E, int64_t n_nodes);

/* ---- late-time profiles and the virtual-cathode estimate (Sec. 3) -----
 * Sec. 3 reads the diode state off late-time averaged potential profiles and
 * compares the net transport efficiency with a virtual-cathode transmission
 * estimate (Eq. 9-10).  Sampling rule: after every step n with n >=
 * window_start and (n - window_start) % period == 0, the potential of the new
 * state and, per species, the linear-weight deposit of its particles are added
 * to per-node sums on the device. */

/* Turn sampling on (period >= 1) or off (0) for every instance; clears the
 * sums either way.  The first call with period >= 1 allocates 32 bytes per
 * node.  While on, each step launches one more kernel, which returns at once
 * on steps that are not samples. */
int pic_set_profile_period(pic_handle* h, int64_t period);

/* Averages over the K samples taken so far by one instance, on its
 * n_nodes = n_cells + 1 nodes.  Any output may be NULL.
 *   phi_avg[j]             mean potential, V
 *   density[s*n_nodes + j] mean number density of species s, m^-3: the
 *                          sampled linear weights times the macro weight over
 *                          the node's length (dz inside, dz/2 at electrodes)
 *   counts[s*n_nodes + j]  the exact sums behind density, 2^24 units per
 *                          particle (bit-exact test hook)
 *   *n_samples             K
 * With K = 0 the averages are NaN.  PIC_EINVAL if sampling was never turned
 * on or n_nodes != n_cells + 1.  Synchronises. */
int pic_get_profiles(pic_handle* h, int instance, int64_t n_nodes, double* phi_avg,
                     double* density, int64_t* counts, int64_t* n_samples);

/* Eq. 9-10 of one instance, from the window tallies and the averaged phi. */
typedef struct pic_vc {
    int64_t samples;          /* profile samples behind phi_min */
    double T_emit_eV;         /* k T_wall / e */
    double net_efficiency;    /* Gamma_net / Gamma_emit over the window */
    double phi_vc_eff;        /* Eq. 10: T_emit ln(Gamma_net / Gamma_emit), V; NaN if <= 0 */
    double phi_min;           /* minimum of the averaged phi over the nodes
                                 j <= floor(near_fraction * n_cells) (at least
                                 nodes 0 and 1), V; <= 0 since phi_0 = 0 */
    double z_min;             /* position of the first node holding it, m */
    double eta_vc;            /* Eq. 9 at phi_min, wall phi_w = 0: exp(phi_min / T_emit) */
} pic_vc;

/* near_fraction in (0, 1].  PIC_EINVAL without profile samples.
 * Synchronises. */
int pic_virtual_cathode(pic_handle* h, int instance, double near_fraction, pic_vc* out);

/* ---- checkpoint / resume ---------------------------------------------
 * The paper's production runs take 4.5e6 steps (Sec. 3); a run can be cut
 * into pieces.  A checkpoint holds the whole handle: every instance's live
 * particles in array order, step index, id counter, window tallies and
 * profile sums.  Every random draw is keyed by (seed, species, particle id,
 * step) and the charge deposit is exact integer arithmetic, so a handle that
 * loads a checkpoint continues bit for bit as the uninterrupted run would,
 * given the same launch shape (pic_tune).  The byte format is private to the
 * library, versioned, and checked on load. */

/* Bytes pic_save needs for the current state.  Synchronises. */
int pic_checkpoint_bytes(pic_handle* h, size_t* bytes);

/* Write the state to a host buffer of `bytes` bytes; *written (may be NULL)
 * receives the size used.  PIC_ECAPACITY if the buffer is too small (nothing
 * written).  Synchronises. */
int pic_save(pic_handle* h, void* host_buf, size_t bytes, size_t* written);

/* Replace the state of a handle with a checkpoint of `bytes` bytes (at least
 * what pic_save wrote).  The handle must have been
 * created with the same instance count, configurations (every pic_config
 * field but size and reserved0) and resolved capacities; otherwise, or if
 * the buffer is not a checkpoint of this library version, PIC_EINVAL and the
 * handle is unchanged.  Profile sampling takes the checkpoint's period.
 * Synchronises. */
int pic_load(pic_handle* h, const void* host_buf, size_t bytes);

/* Set the step index of every instance (Philox counters use it). */
int pic_set_step(pic_handle* h, int64_t step);

/* Change launch knobs (see pic_tuning). */
int pic_tune(pic_handle* h, const pic_tuning* t);

/* Sort every species of every instance by cell now (stable counting sort). */
int pic_sort(pic_handle* h);

/* Wait for the stream; return the first sticky error. */
int pic_synchronize(pic_handle* h);

/* Text of the first CUDA failure on this handle ("" if none): the library
 * call site and cudaGetErrorString.  Owned by the handle. */
const char* pic_last_error(const pic_handle* h);

/* Stable sort of one particle set by cell, allocating nothing.
 *
 * The paper has no counterpart: this is a library service for callers that
 * may not allocate device memory -- code that runs after a fixed memory
 * budget has been reserved (a real-time loop, an arena-managed host
 * application, a plugin inside another framework's memory pool), where a
 * cudaMalloc could fail, block or synchronise the device at the wrong time.
 * The caller passes inputs and outputs; the scratch (a (cell, chunk)
 * histogram) is a fixed 4 MiB device array inside this library that every
 * GPU loading the library holds until the process exits.
 *
 * z..id: n input particles (device); z_out..id_out: n outputs (device), not
 * aliasing the inputs.  Output = input stably sorted by the fixed-point cell
 * rule with Nz = n_cells, L = gap_m (the same order as pic_sort).  Enqueued
 * on cuda_stream.  Limits: n <= 2^31 - 1 (positions are 32-bit), n_cells *
 * ceil(n / 8192) <= 2^20 (for example 4.19M particles over 2048 cells) and
 * 1 <= n_cells <= 4096; beyond them it returns PIC_ECAPACITY (PIC_EINVAL for
 * a bad n_cells) without launching anything.  The first call on each
 * device sets up that device (it looks up the scratch's device address and
 * raises a kernel attribute) and should come before any stream capture.
 * Every call shares the one scratch array and overwrites all of it that it
 * reads: calls that overlap on the GPU (other streams, other threads) race
 * and must be serialised by the caller.  No cudaMalloc, cudaFree or
 * allocating library routine is called. */
int pic_sort_by_cell_static(const float* z, const float* vx, const float* vy, const float* vz,
                            const uint32_t* id, int64_t n, int32_t n_cells, double gap_m,
                            float* z_out, float* vx_out, float* vy_out, float* vz_out,
                            uint32_t* id_out, void* cuda_stream);

/* ---- surrogate MLP (learned extension) -------------------------------
 * 5 -> 128 -> 128 -> 128 -> 4 multilayer perceptron with exact-erf GELU on
 * the hidden layers and a linear output, mapping normalised diode settings
 * (emission flux, wall temperature, neutral density, gap, bias) to the
 * Sec. 2.3 / Eq. 4 diagnostics (backflow ratio, net transport efficiency,
 * collection efficiency, cathode energy metric).  The paper has no such
 * model; it places the PIC runs of a flux scan.  Parameters are one flat
 * FP32 master vector of PIC_MLP_PARAMS entries: for each layer W (n_out x
 * n_in, row-major) then b (n_out); the forward/backward read a bfloat16 copy
 * of it (same indices) for the weights and the FP32 biases, with FP32
 * activations and accumulation.  All pointers are device memory; work is
 * enqueued on cuda_stream; results are deterministic. */
#define PIC_MLP_PARAMS 34308

/* Scratch bytes pic_mlp_grad / pic_mlp_train_step need for a batch. */
size_t pic_mlp_scratch_bytes(int64_t batch);
/* w_bf16[p] = bfloat16(master[p]), round to nearest even. */
int pic_mlp_cast_bf16(const float* master, uint16_t* w_bf16, void* cuda_stream);
/* y[batch x 4] = MLP(x[batch x 5]). */
int pic_mlp_forward(const float* master, const uint16_t* w_bf16, const float* x, int64_t batch,
                    float* y, void* cuda_stream);
/* Mean squared error over the batch and the 4 outputs against t[batch x 4]
 * (*loss, device) and its gradient w.r.t. the parameters (grad[PIC_MLP_PARAMS]). */
int pic_mlp_grad(const float* master, const uint16_t* w_bf16, const float* x, const float* t,
                 int64_t batch, float* grad, float* loss, float* scratch, size_t scratch_bytes,
                 void* cuda_stream);
/* One Adam step (Kingma & Ba) at step >= 1 on the master, moments adam_m,
 * adam_v, refreshing w_bf16; *loss (device, may be NULL) gets the batch MSE
 * before the update. */
int pic_mlp_train_step(float* master, uint16_t* w_bf16, float* adam_m, float* adam_v,
                       int64_t step, float lr, float beta1, float beta2, float eps,
                       const float* x, const float* t, int64_t batch, float* loss, float* scratch,
                       size_t scratch_bytes, void* cuda_stream);

/* Release the handle and all device state it owns.  NULL is ignored. */
void pic_destroy(pic_handle* h);
/* Static description of a PIC_E* code. */
const char* pic_strerror(int code);
int pic_abi_version(void);
/* sizeof of the ABI structs for foreign bindings: 0 pic_config, 1 pic_tuning,
 * 2 pic_diag, 3 pic_profile, 4 pic_vc; 0 for anything else. */
size_t pic_sizeof(int which);

#ifdef __cplusplus
}
#endif
#endif /* PIC_H */
