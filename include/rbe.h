/*
 * librbe -- random batch Ewald (RBE) k-space forces, energy and virial on one GB300 GPU.
 *
 * The method (Liang, Tan, Hong, Jin, Xu, Li, "A random batch Ewald method for charged
 * particles in the isothermal-isobaric ensemble"): N charges q_i at r_i in a periodic
 * rectangular box h = diag(l_x, l_y, l_z) (Sec. 4.1, App. C).  Each evaluation draws P
 * frequencies k = 2 pi m / l (m in Z^3 \ {0}) i.i.d. from the discrete Gaussian
 * P(k) = exp(-|k|^2/4a) / S, S = H_x H_y H_z - 1 (Sec. 4.2 Eqs. (S), (psf),
 * (probexpression); App. C item 1), forms rho(k) = sum_i q_i e^{i k.r_i}, and returns
 *   forces   F_i = -sum_l (S/P) (4 pi q_i k_l / (V |k_l|^2)) Im(e^{-i k_l.r_i} rho(k_l))
 *                                                                  Sec. 4.2 Eq. (appforce)
 *   virial   W = (2 pi / V) sum_l (S/P) |rho_l|^2/|k_l|^2 [I - 2 (1/|k_l|^2 + 1/4a) k_l k_l]
 *            (energy units: the k-space pressure tensor is W / V)   App. C Eq. (pressuretensorflexible);
 *            tr(W)/(3V) is P_2* of Sec. 4.2 Eq. (apppress)
 *   energy   E_k = (2 pi / V) sum_l (S/P) |rho_l|^2/|k_l|^2 and E_self = -sqrt(a/pi) sum_i q_i^2
 *            (importance-weighted form of Sec. 4.1 Eq. (U1fourier))
 * Units are Gaussian (U = 1/2 sum q_i q_j / r): multiply by the caller's Coulomb constant.
 *
 * Conventions for every call:
 *  - Ownership: the caller owns every buffer it passes; nothing is freed across the
 *    boundary.  The context owns only its scratch and tables.
 *  - Device pointers must be CUDA device (or managed) memory of the current device,
 *    8-byte aligned; host pointers are ordinary host memory.
 *  - Device outputs are written asynchronously on the context's stream (rbe_set_stream);
 *    calls taking host buffers synchronise that stream before returning.
 *  - Every call validates all arguments before any launch and returns without side
 *    effects on RBE_EINVAL.  rbe_last_error() gives a message for the last failure.
 *  - Errors detected on the device (a sample that stayed at m = 0 for 2^20 redraws, a
 *    non-finite rho) are latched in a device status word and returned by the next
 *    synchronising call (rbe_sync, rbe_sample_k, the *_host calls).
 *  - One context per host thread; calls on one context are not thread-safe.
 */
#ifndef RBE_H
#define RBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rbe_ctx_s* rbe_ctx;

typedef enum {
    RBE_OK = 0,
    RBE_EINVAL = 1,      /* bad argument: null/misaligned pointer, N < 0, P < 1, alpha <= 0, box <= 0 ... */
    RBE_ENOMEM = 2,      /* device or host allocation failed */
    RBE_ECUDA = 3,       /* a CUDA runtime call or launch failed (message in rbe_last_error) */
    RBE_ETIMEOUT = 4,    /* a bounded device-side wait gave up (the persistent batched launch's grid
                            barriers); no other call waits on the device */
    RBE_ENONFINITE = 5,  /* rho(k) or an output became NaN/Inf (non-finite inputs) */
    RBE_ESTATE = 6,      /* call not valid in the context's current state */
    RBE_ESAMPLE = 7      /* a frequency stayed m = 0 after 2^20 redraws (alpha l^2 far too small) */
} rbe_status;

typedef enum {
    RBE_FP64 = 0,        /* phases, sincos and accumulation in FP64 */
    RBE_FP32_PHASE = 1   /* exact 32-bit fixed-point phase m.s mod 1, FP32 sine and cosine (rho pass)
                            and one FP32 sine of the phase shifted by arg rho (force pass),
                            float-float sums across tiles */
} rbe_precision;

typedef enum {
    RBE_RHO_FP64 = 0,    /* FP32-phase path: rho accumulated per pair in FP64 */
    RBE_RHO_COMP32 = 1,  /* FP32-phase path: compensated FP32 summation within a staged tile (FP32
                            partial sums of 16 consecutive particles added with Kahan's
                            compensation: a rounding error that does not grow with the particle
                            count, to first order at most 17 eps sum |q| per tile), float-float
                            (about 48 bits) across tiles (default) */
    RBE_RHO_FP32 = 2     /* FP32-phase path: plain FP32 within a staged tile, float-float across (faster;
                            outside the compensated-or-FP64 rule of the default) */
} rbe_rho_accum;

/* Create a context for box lengths box[3] (> 0), splitting parameter alpha (> 0, Sec. 4.1),
 * batch size P (1 <= P <= 65536, Sec. 4.2) and the Philox key seed.  Allocates the
 * context's device scratch on the current CUDA device.  *out is set only on RBE_OK.
 * The box must satisfy pi^2 / (alpha l^2) <= 600 on every axis (otherwise S underflows
 * and the frequency distribution is degenerate): RBE_EINVAL. */
rbe_status rbe_create(const double box[3], double alpha, int32_t P, uint64_t seed, rbe_ctx* out);

/* Free the context and its device scratch (synchronises its stream first).  NULL is a no-op. */
rbe_status rbe_destroy(rbe_ctx ctx);

/* Set the CUDA stream (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream)
 * on which all later device work of this context runs.  NULL = the legacy default stream.
 * The context's scratch is allocated in stream order; switching streams first waits for the
 * old stream. */
rbe_status rbe_set_stream(rbe_ctx ctx, void* stream);

/* Replace the Philox key used by later calls (sampling and NPT noise). */
rbe_status rbe_set_seed(rbe_ctx ctx, uint64_t seed);

/* Select the arithmetic: precision in rbe_precision, rho_accum in rbe_rho_accum
 * (rho_accum is ignored on the FP64 path).  A new context runs RBE_FP64 with RBE_RHO_COMP32.
 * On the FP32-phase path every accumulation widens rho(k) to FP64 before the per-frequency
 * energy and virial terms, which are formed and summed in FP64. */
rbe_status rbe_set_precision(rbe_ctx ctx, int32_t precision, int32_t rho_accum);

/* Frequency samplers (Sec. 4.3).  EXACT (default): i.i.d. draws from the discrete Gaussian of
 * Eq. (probexpression) by per-axis inverse CDF.  OFFLINE: the paper's offline approach, Gaussian
 * z drawn independently of the box (Philox stream 3, Marsaglia's polar method), m_j =
 * rint(z_j sqrt(alpha l_j^2 / (2 pi^2))), redrawn while m = 0; the weights stay S/P, so the
 * rounding is a systematic bias (the paper notes it; the estimator is no longer unbiased).
 * MH: the paper's online approach, one Metropolis--Hastings step per frequency slot and call,
 * from the slot's previous m, with the offline draw as an independence proposal (its mass per
 * integer the Gaussian mass of [m - 1/2, m + 1/2)) and the discrete Gaussian on Z^3 \ {0} as
 * the target; acceptance uniform from Philox stream 4.  The chain state lives in the context
 * (one slot per frequency, sized for the context's P); every rbe_set_sampler call resets it, and
 * a reset slot starts from the EXACT draw of its next step.  Every floating-point step that
 * decides an integer is a separately rounded IEEE operation written out in the library (own
 * logarithm, erfc and exponential), so the draws match the oracle bit for bit.  Applies to
 * rbe_sample_k, rbe_kspace_forces_virial(_host) and rbe_npt_step; the batched API and
 * rbe_sample_k_noalloc always use EXACT.  A CUDA graph captured earlier keeps the sampler it
 * was captured with.  RBE_EINVAL for an unknown sampler. */
typedef enum { RBE_SAMPLER_EXACT = 0, RBE_SAMPLER_OFFLINE = 1, RBE_SAMPLER_MH = 2 } rbe_sampler;
rbe_status rbe_set_sampler(rbe_ctx ctx, int32_t sampler);

/* A separate batch of Ptilde frequencies for the pressure (Eq. (apppress) with its own p~; the
 * paper notes that the force and pressure samples may differ).  0 (default): energy and virial
 * come from the force batch.  Ptilde > 0: every sampling step draws P + Ptilde frequencies (the
 * force batch in slots [0, P), the same draws as without a pressure batch; the pressure batch in
 * slots [P, P + Ptilde), Philox slot counters continuing past P); forces use the force batch with
 * weights S/P, the virial and the energy (E_k, E_self) the pressure batch with weights S/Ptilde.
 * Applies to rbe_kspace_forces_virial(_host) and rbe_npt_step (its pressure and energies); with
 * RBE_SAMPLER_MH the chain grows to P + Ptilde slots and restarts from the exact draw.  The host-
 * buffer call then copies in, evaluates and copies out without pipelining.  rbe_sample_k still
 * returns the force batch; rbe_get_rho returns the pressure batch's rho.  RBE_EINVAL unless
 * 0 <= Ptilde <= 2^20. */
rbe_status rbe_set_pressure_batch(rbe_ctx ctx, int32_t Ptilde);

/* Sample reuse for the NPT step (Sec. 4.3, the strategy that updates the samples every M
 * steps).  M = 1 (default): every step draws its own frequencies.  M > 1: at a step s with
 * s mod M = 0 the sampler draws M batches at once from that step's box (counter step s, batch i
 * in slots [i (P + Ptilde), (i + 1) (P + Ptilde))), kept on the device; step s + i evaluates
 * batch i with the wave vectors k = 2 pi m / l and the weights S/P (S/Ptilde) of its own box.
 * Batch 0 is the ordinary draw of step s; the later batches carry the stale-box error the paper
 * describes.  Applies to rbe_npt_step only.  RBE_EINVAL unless 1 <= M <= 1024, or with the
 * Metropolis--Hastings sampler (the two exclude each other). */
rbe_status rbe_set_sample_reuse(rbe_ctx ctx, int32_t M);

/* RBE k-space forces, virial and energy in a general (triclinic) cell (App. C, the fully
 * flexible cell).  h: host 3x3, row-major, the cell vectors as COLUMNS (h[3 i + j] = component i
 * of vector j), det h > 0; positions any real (r = h s, s scaled coordinates); wave vectors
 * k = 2 pi h^{-T} m, the phase k.r = 2 pi m.s.  Frequencies: the law exp(-pi^2 m^T G m / alpha)
 * (G = h^{-1} h^{-T}) does not factorise, so each slot runs a Metropolis--Hastings chain (the
 * paper's suggestion): an independence proposal from the exact product of per-axis discrete
 * Gaussians with lengths l_j = sqrt(lambda) |a_j| (|a_j| the cell vector lengths, lambda =
 * max_j (1 + sum_{k != j} |cos theta_jk|), so the ratio of target to proposal is bounded and a
 * rectangular cell proposes the target itself), Philox stream 0 as the exact sampler with these
 * lengths; acceptance with O(m) = (pi^2/alpha) m^T G m - sum_j (pi^2/(alpha l_j^2)) m_j^2: m'
 * when O(m') <= O(m), else when u < exp(O(m) - O(m')), u from stream 5 (l, 0, step_lo,
 * (5 << 24) | step_hi24).  The chain state is the context's (P slots); a slot at m = 0 (first
 * call, or after rbe_set_sampler) starts from the proposal; m matches the oracle bit for bit.
 * Weights S/P with S = sum_{m != 0} exp(-pi^2 m^T G m / alpha) from the Poisson dual sum
 * (alpha/pi)^{3/2} V sum_n exp(-alpha |h n|^2) - 1.  Outputs as rbe_kspace_forces_virial: forces
 * (device N*3, overwritten), virial (device 9, the full tensor of App. C Eq.
 * (pressuretensorflexible), or NULL), energy (device 2: E_k, E_self, or NULL).  Runs the context's
 * precision (the FP32-phase passes on the scaled coordinates).  Asynchronous; RBE_EINVAL for a
 * singular, non-finite or oversized cell or bad arguments; device errors via rbe_sync. */
rbe_status rbe_kspace_forces_virial_general(rbe_ctx ctx, int64_t N, const double* positions, const double* charges,
                                            const double h[9], uint64_t step, double* forces_out,
                                            double* virial_out, double* energy_out);

/* Replace the box lengths (same validity rule as rbe_create).  The per-axis sampling
 * tables are rebuilt on the device at the next evaluation. */
rbe_status rbe_set_box(rbe_ctx ctx, const double box[3]);

/* Draw the batch of one step (Sec. 4.2-4.3; App. C item 1) into HOST memory:
 * m_out[P][3] int32 row-major (may be NULL) and S (may be NULL).  Sample l depends only
 * on (seed, step, l): Philox-4x32-10 with key (seed_lo, seed_hi) and counter
 * (l, 2*attempt + half, step_lo32, step_hi24); three 53-bit uniforms; per-axis inverse
 * CDF of exp(-c m^2), c = pi^2/(alpha l^2), truncated at |m| <= ceil(sqrt(60 ln2 / c));
 * redraw (attempt + 1) while m = 0.  step < 2^56.  Synchronous. */
rbe_status rbe_sample_k(rbe_ctx ctx, uint64_t step, int32_t* m_out, double* S_out);

/* One RBE k-space evaluation on DEVICE buffers (Sec. 4.2 Eqs. (appforce), (apppress);
 * App. C Eq. (pressuretensorflexible)).
 *   N           number of particles, N >= 0 (N = 0 gives zero outputs)
 *   positions   device, N*3 double, row-major (x, y, z); need not be wrapped into the box
 *   charges     device, N double
 *   step        Philox counter of the batch: the same step gives the same m as rbe_sample_k
 *   forces_out  device, N*3 double, overwritten with the k-space force only
 *   virial_out  device, 9 double, row-major 3x3 W in energy units (may be NULL)
 *   energy_out  device, 2 double {E_k, E_self} (may be NULL)
 * Asynchronous on the context's stream. */
rbe_status rbe_kspace_forces_virial(rbe_ctx ctx, int64_t N, const double* positions,
                                    const double* charges, uint64_t step, double* forces_out,
                                    double* virial_out, double* energy_out);

/* The same evaluation with float32 positions and charges: xyzq is device memory holding one
 * float4 (x, y, z, q) per particle, N*4 floats, 16-byte aligned.  Each coordinate is widened to
 * the double it equals (exactly) and enters the same exact fixed-point phase as the FP64 input,
 * so the result is the evaluation of the float-rounded positions and charges: the error of the
 * input's rounding is separate from the path's own.  Needs the RBE_FP32_PHASE precision
 * (RBE_EINVAL otherwise); the context's rho accumulation applies.  Other arguments as
 * rbe_kspace_forces_virial.  Asynchronous. */
rbe_status rbe_kspace_forces_virial_xyzq(rbe_ctx ctx, int64_t N, const float* xyzq, uint64_t step,
                                         double* forces_out, double* virial_out, double* energy_out);

/* The same evaluation on HOST buffers: copies positions and charges to context-owned
 * device buffers, evaluates, copies forces, virial and energy back, synchronises the
 * stream and returns any latched device error.  forces_out may be NULL.  On the FP32-phase
 * path with N >= 2^17 the copies are pipelined with the passes: the particles go in two
 * groups (four from N >= 2^19: an eighth, three eighths, three eighths and an eighth), each
 * evaluated by full-GPU passes of its own, so that a group's copy in overlaps the previous
 * group's rho pass and its forces' copy out overlaps the next group's force pass.
 * The sums then run over a different chunk partition: the results agree with
 * rbe_kspace_forces_virial to FP32 rounding and are reproducible run to run.  Page-locked
 * host buffers let the copies overlap fully. */
rbe_status rbe_kspace_forces_virial_host(rbe_ctx ctx, int64_t N, const double* positions,
                                         const double* charges, uint64_t step, double* forces_out,
                                         double* virial_out, double* energy_out);

/* Weighted evaluation on a caller-given frequency list (no sampling): the estimator of
 * rbe_kspace_forces_virial with S/P replaced by weights[l] for frequency m[l].  With
 * every m of a cube |m_theta| <= kmax and weights exp(-|k|^2/4a) this is the plain
 * Ewald k-space sum of Sec. 4.1 Eqs. (U1fourier), (force).
 *   K          number of frequencies, 1 <= K <= 2^24
 *   m          device, K*3 int32 (no all-zero row: RBE_EINVAL is not checked on the
 *              device; a zero row yields a non-finite result latched as RBE_ENONFINITE)
 *   weights    device, K double
 * Other arguments as rbe_kspace_forces_virial.  Asynchronous. */
rbe_status rbe_kspace_weighted(rbe_ctx ctx, int64_t N, const double* positions, const double* charges,
                               int32_t K, const int32_t* m, const double* weights, double* forces_out,
                               double* virial_out, double* energy_out);

/* Copy the last evaluation's rho(k_l) (interleaved re, im; 2*P doubles, or 2*K after a
 * weighted call) into HOST memory.  Synchronous. */
rbe_status rbe_get_rho(rbe_ctx ctx, double* rho_out, int32_t capacity);

/* Measurement support (no counterpart in the paper).  With timing enabled the context
 * records CUDA events on its stream around the kernels of each evaluation;
 * rbe_get_kernel_times waits for the last evaluation and returns the durations in ms of
 * {sampling, rho pass, rho reduction + energy/virial, force pass}. */
rbe_status rbe_set_kernel_timing(rbe_ctx ctx, int32_t enable);
rbe_status rbe_get_kernel_times(rbe_ctx ctx, float ms_out[4]);

/* Throughput probe of one GPU pipe on the current device, in operations per second:
 * kind 0 = MUFU sine (sin.approx.f32), 1 = FP32 FMA, 2 = FP64 FMA; `iters` rounds of 8
 * independent operations per thread over 8 x 256-thread blocks per SM, best of three.
 * Synchronous, legacy default stream.  The measured denominators of the roofline. */
rbe_status rbe_measure_pipe(int32_t kind, int32_t iters, double* ops_per_s);

/* Allocation-free sampling (the paper has no counterpart: this serves callers that cannot
 * allocate device memory when they need a batch -- an MD engine that sized one device pool at
 * start-up and allows no allocation afterwards, a plugin inside an application that owns all
 * device memory, or a loop that must not call cudaMalloc because a device allocation can
 * synchronise the whole device).  Draws the same batch as rbe_sample_k for (box, alpha, P,
 * seed, step) without a context and without allocating: no cudaMalloc, no cudaFree, no
 * allocating library routine.
 *   box, alpha, P, seed, step  as rbe_create / rbe_sample_k
 *   m_out    device, P*3 int32 row-major (4-byte aligned), written
 *   S_out    device, 1 double (8-byte aligned), written with S = H_x H_y H_z - 1
 *   stream   cudaStream_t to run on (NULL = legacy default stream)
 * Scratch: a fixed file-scope device array of 192 KB (three tables of up to 8191 entries and a
 * status word) that every GPU which loads the library holds until the process exits.  Boxes
 * that need more than 4094 frequencies per axis (2 sqrt(alpha) l > ~4094) are rejected with
 * RBE_EINVAL ("too large for the fixed scratch"); use rbe_sample_k for those.
 * Every call shares the array, which keeps the last call's contents (the status word is
 * cleared at the start of each call); calls that overlap on the GPU -- on different streams
 * or from different host threads -- race on it and must be serialised by the caller.
 * Every call looks up the array's device address (cudaGetSymbolAddress, a host-side query that
 * allocates nothing) in the CUDA context current on the calling thread, so a caller that
 * switches contexts or resets the device gets the address of the array in the context it runs
 * in.  Not usable during stream capture: every call ends with a copy of the status word into
 * host memory and a synchronisation of `stream`, which a capturing stream refuses.  A frequency
 * that stayed m = 0 after 2^20 redraws returns RBE_ESAMPLE.
 * Messages for failures are returned by rbe_last_error(NULL). */
rbe_status rbe_sample_k_noalloc(const double box[3], double alpha, int32_t P, uint64_t seed, uint64_t step,
                                int32_t* m_out, double* S_out, void* stream);

/* Synchronise the context's stream and return (and clear) any latched device error. */
rbe_status rbe_sync(rbe_ctx ctx);

/* ---------------------------------------------------------------------------------
 * Langevin NPT (Sec. 3.2 Eq. (24); Sec. 3.3 splitting
 *   V^p/2, R^p/2, V/2, R/2, O^p, O, R/2, V/2, [forces, P_ins], R^p/2, V^p/2
 * with the R and R^p flows solved exactly for frozen strain rates and exact
 * Ornstein--Uhlenbeck steps O, O^p).  Forces: the context's RBE k-space estimator (batch of
 * the step index, Sec. 4.2) times qqr2e, plus the nearest-image real space within rc:
 * qqr2e q_i q_j erfc(sqrt(alpha) r)/r + 4 eps ((sigma/r)^12 - (sigma/r)^6) (Sec. 4.1-4.2).
 * Units: A, ps, g/mol, kJ/mol, e; momenta in g/mol A/ps (dp/dt = 100 F for F in kJ/mol/A);
 * pressure in kJ/mol/A^3.  Noise: Philox-4x32-10 with the context's seed, counters
 * (i, 0, step_lo, (1 << 24) | step_hi24) for particle i and (0, 0, step_lo, (2 << 24) |
 * step_hi24) for the cell, 32-bit uniforms (w + 1/2) 2^-32 and Box--Muller (the particle
 * normals in FP32 arithmetic on the FP32-phase path, FP64 otherwise).
 *
 * barostat 1, isotropic: the volume V with momentum p_V (kJ/mol ps/A^3) and mass M_V
 *   (kJ/mol ps^2/A^6); eps = p_V / (3 M_V V) on every axis; P_ins = (sum p^2/m + W_k + W_r) / (3V)
 *   (Sec. 4.1 Eq. (pressurecubic)); the box scales by (V'/V)^(1/3); the cell normal z[0].
 * barostat 2, rectangular cell with anisotropic fluctuation (appendix): the edges l_j with
 *   momenta pc_j (kJ/mol ps/A) and masses M_cell[j] (kJ/mol ps^2/A^2); eps_j = pc_j / (M_j l_j);
 *   dpc_j/dt = V ((P_ins)_jj - P) / l_j - gamma_V pc_j + noise with (P_ins)_jj =
 *   (sum_i p_ij^2/m_i + W_jj) / V, W_jj the diagonal of the k-space and real-space virials;
 *   V/2 moves l_j by (dt/2) pc_j / M_j; slot j takes the cell normal z[j].
 * barostat 3, semi-isotropic at constant surface tension (appendix): the area A = l_x l_y
 *   (l_x = l_y required) with momentum pc_0 (kJ/mol ps/A^2) and mass M_cell[0]
 *   (kJ/mol ps^2/A^4), the height L = l_z with momentum pc_2 and mass M_cell[2];
 *   eps_x = eps_y = pc_0 / (2 M_A A), eps_z = pc_2 / (M_L L); dpc_0/dt = L (P_A - P) + noise,
 *   P_A = ((P_ins)_xx + (P_ins)_yy)/2 + gamma0 / L; dpc_2/dt = A ((P_ins)_zz - P) + noise;
 *   l_x = l_y = sqrt(A) after each move; the normals z[0] and z[2].
 * gamma_V is the friction of every cell variable. */
typedef struct {
    double dt;        /* time step, ps */
    double kT;        /* k_B T, kJ/mol */
    double P_ext;     /* external pressure, kJ/mol/A^3 */
    double gamma;     /* particle friction, 1/ps */
    double gamma_V;   /* cell friction, 1/ps */
    double M_V;       /* isotropic piston mass, kJ/mol ps^2/A^6 (> 0 when barostat == 1) */
    double rc;        /* real-space cutoff, A (rc <= box/2 on every axis) */
    double qqr2e;     /* Coulomb constant, kJ/mol A/e^2 */
    double lj_sigma;  /* A */
    double lj_eps;    /* kJ/mol; 0 disables the Lennard-Jones term */
    double max_disp;  /* cap on the peculiar displacement |(p/m) dt| per step in A, split over the two
                         R/2 sub-steps; the dilation with the cell is not capped; 0 = none */
    int32_t kspace;   /* 1: RBE k-space forces and virial */
    int32_t real;     /* 1: real-space forces and virial */
    int32_t noise;    /* 1: Langevin noise in O and O^p */
    int32_t barostat; /* 0: the box is fixed; 1: isotropic; 2: anisotropic rectangular;
                         3: semi-isotropic with surface tension */
    double skin;      /* A.  0: the real-space pairs come from a cell search every step.  > 0: from
                         a neighbour list of radius rc + skin, rebuilt on the device when the largest
                         displacement since the last build and the box change could have brought an
                         unlisted pair within rc (the same pairs either way) */
    double M_cell[3]; /* barostat 2: masses of l_x, l_y, l_z (> 0); barostat 3: M_A in [0] and M_L
                         in [2] (> 0), [1] unused */
    double gamma0;    /* barostat 3: surface tension times the number of surfaces, kJ/mol/A^2 */
} rbe_npt_params;

/* Number of doubles of the device cell-state block:
 *   [0..2]  l_x, l_y, l_z            [3]  p_V (barostat 1)
 *   [4]     W, trace of the virial at the current positions (k-space x qqr2e + real space)
 *   [5]     sum p^2/m / 100 (= 2K)   [6]  P_ins = (2K + W) / (3V)
 *   [7]     E_k (k-space incl. self, x qqr2e)   [8] E_coul (real space)   [9] E_lj
 *   [10]    V                        [11] step index (64-bit integer bits)
 *   [12..14] cell momenta of barostats 2 and 3 (pc_x, pc_y, pc_z, or p^A, 0, p^L)
 *   [16..18] W_xx, W_yy, W_zz        [19..21] sum_i p_ij^2/m_i / 100 per axis
 *   [22..24] (P_ins)_xx, (P_ins)_yy, (P_ins)_zz   ([16..24] with barostat 2 and 3 only)
 * the rest reserved. */
#define RBE_CELL_DOUBLES 32

/* One replica; every buffer is the caller's device memory.  `step` is the next step index
 * (the Philox counter of its RBE batch and noise); rbe_npt_step advances it. */
typedef struct {
    int64_t N;
    double* pos;          /* device N*3, wrapped into [0, l) after every step */
    double* mom;          /* device N*3 */
    double* force;        /* device N*3: forces at pos, kJ/mol/A (kept between steps) */
    const double* charge; /* device N, e */
    const double* mass;   /* device N, g/mol */
    double* cell;         /* device RBE_CELL_DOUBLES (box in cell[0..2] must be set by the caller) */
    uint64_t step;        /* host */
    rbe_npt_params params;
} rbe_system;

/* Forces, virial and energies at the current state, with the RBE batch of index `batch`;
 * fills sys->force, cell[4..10] and, with barostat 2 or 3, cell[16..24] (the cell momenta
 * p_V and cell[12..14] are kept).  Call once before the first step.
 * Reads the initial box back (synchronises the context's stream) and sizes the per-axis
 * tables and the cell list for box edges up to twice the initial ones; a step whose box
 * leaves that range, or breaks rc <= l/2 with real space on, is flagged on the device and
 * reported as RBE_ESTATE by the next rbe_sync.  Asynchronous otherwise.  RBE_EINVAL for bad
 * pointers or parameters. */
rbe_status rbe_npt_init(rbe_ctx ctx, rbe_system* sys, uint64_t batch);

/* Advance nsteps >= 1 steps (Sec. 3.3); asynchronous on the context's stream; sys->step
 * advances by nsteps.  The context's box is not used: each step rebuilds the sampling tables
 * from the device box in sys->cell.  The step index also lives on the device (cell[11], as
 * 64-bit integer bits, set by rbe_npt_init and advanced by every step), so the launches of
 * one call may be captured once in a CUDA graph and replayed for later steps. */
rbe_status rbe_npt_step(rbe_ctx ctx, rbe_system* sys, int32_t nsteps);

/* ---------------------------------------------------------------------------------
 * Langevin NPT of rigid 3-site water (the paper's water runs keep molecules rigid, Sec. 5.1).
 * sys->N counts sites, ordered O, H, H per molecule (N a multiple of 3); charges and masses per
 * site; sys->params as for rbe_npt_step with barostat 0 or 1, skin 0, and the Lennard-Jones
 * parameters acting between oxygens only.  Each molecule's centre of mass follows the isotropic
 * Langevin NPT equations (Sec. 3.2, splitting of Sec. 3.3) with the molecule's mass and total
 * force, the cell scaling the centres only; the internal motion is constrained: R^p/2 kicks the
 * internal momenta by (dt/2) 100 (F_i - m_i F/M), R/2 moves the offsets freely and the SHAKE
 * equations restore the O-H, O-H and H-H distances (corrections along the old separations, solved by
 * Newton's method on the three multipliers until every |r^2 - d^2| <= tol d^2; the displacement
 * enters the momenta), O acts on every site (Philox stream 1 at the site index),
 * and after R^p/2, R/2 and O the momenta are projected onto the velocity constraints (RATTLE).
 * The barostat sees (sum_I |P_I|^2 / M_I / 100 + W_mol) / (3V), W_mol = W - sum_i F_i . d_i (d_i
 * the site's offset from its molecule's centre).  Forces: the context's RBE k-space over all sites
 * times qqr2e, minus -qqr2e q_i q_j erf(sqrt(alpha) r)/r for the three site pairs of each
 * molecule, plus erfc Coulomb between sites of different molecules within rc and LJ between
 * oxygens (FP64, whatever the context's precision; the k-space follows it).  Cell block as
 * rbe_npt_step's isotropic one (cell[4] = W_mol, cell[5] = the centres' 2K, cell[6] the molecular
 * P_ins), plus cell[25] = the exclusion energy.  Molecules are made whole from their oxygen by
 * the nearest image; after every step a molecule moves by the lattice vector that brings its
 * oxygen into the box.  A molecule whose constraint solve does not converge within
 * shake_max_iter iterations is flagged (RBE_ESTATE at the next rbe_sync). */
typedef struct {
    double d_OH;          /* O-H distance, A */
    double d_HH;          /* H-H distance, A */
    double shake_tol;     /* relative tolerance of |r^2 - d^2| / d^2, > 0 */
    int32_t shake_max_iter; /* constraint-solve iterations per molecule and R/2 at most, >= 1 */
    int32_t pad;
} rbe_water_params;

/* As rbe_npt_init and rbe_npt_step for rigid water (the same scratch; the context serves one
 * of the NPT, flexible-cell and water systems at a time). */
rbe_status rbe_water_init(rbe_ctx ctx, rbe_system* sys, const rbe_water_params* wp, uint64_t batch);
rbe_status rbe_water_step(rbe_ctx ctx, rbe_system* sys, const rbe_water_params* wp, int32_t nsteps);

/* ---------------------------------------------------------------------------------
 * Langevin NPT with a fully flexible cell (App. A, the fully flexible cells; the k-space of
 * App. C in a general cell).  The cell h is 3x3, row-major, with the cell vectors a, b, c as its
 * columns (r = h s for scaled coordinates s) and det h > 0; its momenta p^h (kJ/mol ps/A) and
 * masses M (kJ/mol ps^2/A^2) have one entry per entry of h.  With A = (dh/dt) h^{-1}:
 *   dr/dt = p/m + A r,   dp/dt = 100 F - A^T p - gamma p + sqrt(2 gamma 100 kT m) xi,
 *   dh/dt = p^h / M (entrywise),
 *   dp^h/dt = (Kt + W - (P V + chi kT) I) h^{-T} - gamma_h p^h + sqrt(2 gamma_h kT M) xi,
 * Kt = sum_i p_i p_i^T / (100 m_i), W the full virial tensor (k-space x qqr2e plus real space),
 * V = det h.  chi = 2 (d - 1) weights the cells by det(h)^{1-d}, the isobaric ensemble of a
 * flexible cell; without friction and noise the step conserves, to O(dt^2),
 *   H = K + U + P V + chi kT ln V + sum (p^h)^2 / (2 M).
 * Splitting of rbe_npt_step with matrices: R^p/2 (p <- e^{-A^T t} p + t phi(-A^T t) 100 F),
 * R/2 (r <- e^{A t} r + t phi(A t) p/m, the peculiar part capped), V/2 (h += t p^h/M), O^p, O,
 * V^p/2 (p^h += t (Kt + W - (P V + chi kT) I) h^{-T}), with t = dt/2, A frozen over each
 * sub-step and phi(X) = sum_k X^k / (k+1)!.  Cell noise: Philox stream 2 (rbe_npt_step's cell
 * counter) at indices 0 (the diagonal: z[0], z[1], z[2]), 1 and 2 (the off-diagonal entries in
 * row-major order: z1[0..3], z2[0..1]).  Positions are wrapped to s in [0, 1) after every step.
 * k-space: the RBE estimator of rbe_kspace_forces_virial_general (the context's general-cell MH
 * chain, P frequencies, batch = the step index) times qqr2e; the context's sampler, pressure
 * batch and sample reuse settings do not apply.  Real space: the pair terms of rbe_npt_step by
 * the minimum image in scaled coordinates, on a cell list in s or a neighbour list built from
 * it; needs rc (+ skin) <= w_j / 2 for the three widths w_j = V / |a_k x a_l| of the cell. */
typedef struct {
    double dt;        /* ps */
    double kT;        /* kJ/mol */
    double P_ext;     /* kJ/mol/A^3 */
    double gamma;     /* particle friction, 1/ps */
    double gamma_h;   /* cell friction, 1/ps */
    double M[9];      /* cell masses, row-major like h, each > 0 */
    double rc;        /* real-space cutoff, A */
    double qqr2e;     /* Coulomb constant, kJ/mol A/e^2 */
    double lj_sigma;  /* A */
    double lj_eps;    /* kJ/mol; 0 disables the Lennard-Jones term */
    double max_disp;  /* cap on the peculiar displacement per step (split over the two R/2), A; 0 = none */
    double chi;       /* 2 for the flexible-cell ensemble; 0 drops the ln V term */
    int32_t kspace;   /* 1: RBE k-space forces and virial */
    int32_t real;     /* 1: real-space forces and virial */
    int32_t noise;    /* 1: Langevin noise in O and O^p */
    int32_t pad;
    double skin;      /* A.  0: the real-space pairs come from a cell search every step.  > 0: from a
                         neighbour list of radius rc + skin (needs rc + skin <= w_j / 2), rebuilt on
                         the device when the largest displacement since the build and the cell's
                         deformation h h_ref^{-1} could have brought an unlisted pair within rc */
} rbe_flex_params;

/* Doubles of the device cell block of the flexible cell:
 *   [0..8]   h (row-major)         [9..17]  p^h            [18..26] W (full virial tensor)
 *   [27..35] Kt = sum p p^T/(100 m)  [36..44] pressure tensor (Kt + W) / V
 *   [45] E_k (k-space incl. self, x qqr2e)  [46] E_coul (real space)  [47] E_lj  [48] V
 *   [49] H, the extended energy     [50] step index (64-bit integer bits)
 *   [51] neighbour-list builds so far (skin > 0)
 * the rest reserved. */
#define RBE_FLEX_CELL_DOUBLES 64

/* One flexible-cell replica; every buffer is the caller's device memory (8-byte aligned). */
typedef struct {
    int64_t N;
    double* pos;          /* device N*3, wrapped to scaled coordinates in [0, 1) after every step */
    double* mom;          /* device N*3 */
    double* force;        /* device N*3 (kept between steps) */
    const double* charge; /* device N */
    const double* mass;   /* device N */
    double* cell;         /* device RBE_FLEX_CELL_DOUBLES: h and p^h set by the caller */
    uint64_t step;        /* host: the next step index */
    rbe_flex_params params;
} rbe_flex_system;

/* Forces, virial tensor, energies and H at the current state with the RBE batch `batch`;
 * fills sys->force and cell[18..49] (h and p^h are kept).  Call once before the first step.
 * Reads h back (synchronises the context's stream) and sizes the tables and the cell list for
 * cell vectors up to twice as long, and widths up to twice as wide, as the initial ones; a
 * step whose cell leaves that range, or breaks rc <= w_j/2 with real space on, is flagged on
 * the device and reported as RBE_ESTATE by the next rbe_sync.  RBE_EINVAL for bad pointers,
 * parameters or cells. */
rbe_status rbe_flex_init(rbe_ctx ctx, rbe_flex_system* sys, uint64_t batch);

/* Advance nsteps >= 1 steps; asynchronous on the context's stream; sys->step advances by
 * nsteps.  The step index also lives on the device (cell[50]), so the launches of one call may
 * be captured in a CUDA graph and replayed. */
rbe_status rbe_flex_step(rbe_ctx ctx, rbe_flex_system* sys, int32_t nsteps);

/* ---------------------------------------------------------------------------------
 * Batched k-space evaluation: many systems of uneven N (the RBE force, energy and virial of
 * Sec. 4.2 for each) in ONE persistent launch per evaluation: a cooperative grid of resident
 * blocks that runs the five passes (tables, sampling, rho, rho reduction, forces with energy and
 * virial) with a grid barrier between them, each pass a loop over a work list of (item, tile)
 * units.  The barriers wait a bounded time (about a quarter of a second); a barrier that gives up
 * latches RBE_ETIMEOUT, reported by rbe_batch_sync.  FP32-phase path with compensated FP32
 * accumulation (RBE_RHO_COMP32) and FP64 energy and virial terms.  The batch fixes alpha and P;
 * every item brings its own positions, charges, box, Philox key and batch index, and gets the
 * same frequencies m as rbe_sample_k with that key and index; an item's box and index may also
 * live in device memory (box_dev, step_dev: an NPT replica's cell block), read at run time, so a
 * captured graph of the evaluation follows them.  Tile shapes are the batch's
 * (rbe_batch_set_tiles, or chosen by rbe_batch_autotune).  An item's outputs depend only on its
 * own inputs and the tile shapes, not on the other items.  No counterpart in the paper (its runs
 * are single systems). */
typedef struct rbe_batch_s* rbe_batch;

typedef struct {
    int64_t N;             /* >= 1 */
    const double* pos;     /* device N*3 (8-byte aligned), any real positions */
    const double* charge;  /* device N */
    double* forces;        /* device N*3, overwritten with the k-space force */
    double* virial;        /* device 9, row-major, energy units */
    double* energy;        /* device 2 {E_k, E_self}, or NULL */
    double box[3];         /* rectangular box of this item */
    uint64_t seed;         /* Philox key of this item */
    uint64_t step;         /* batch index (< 2^56) */
    const double* box_dev;     /* NULL, or the item's box in device memory (3 doubles, 8-byte aligned):
                                  read by every evaluation (its tables rebuilt each time) instead of
                                  box[], which then only bounds the table size check */
    const uint64_t* step_dev;  /* NULL, or the item's batch index in device memory (read by every
                                  evaluation instead of step) */
    uint32_t* status_dev;      /* NULL, or a device word (4-byte aligned) where this item's device
                                  errors are latched (the bits of a context's status word) instead of
                                  the batch's own, so that a failing item is told apart */
} rbe_batch_item;

/* A batch for up to max_items items with boxes no longer than max_box on any axis (sizes the
 * per-item sampling tables).  RBE_EINVAL for bad parameters; allocates its buffers now. */
rbe_status rbe_batch_create(double alpha, int32_t P, int32_t max_items, double max_box, rbe_batch* out);
rbe_status rbe_batch_destroy(rbe_batch b);
/* Stream of later evaluations (a cudaStream_t; NULL = legacy default); synchronises the old one. */
rbe_status rbe_batch_set_stream(rbe_batch b, void* stream);
/* Tile shapes: rho_k frequency lanes per rho tile (16 to 256; a block of 256 threads runs
 * floor(256 / rho_k) particle sub-streams of the tile, the threads beyond them idle), rho_chunk
 * particles per rho chunk (>= 32), force_block particles per force tile (a positive multiple of
 * 128).  All three 0 restores the defaults (the rho tile that keeps the most lanes busy for this
 * P, chunks of 256, force tiles of 512). */
rbe_status rbe_batch_set_tiles(rbe_batch b, int32_t rho_k, int32_t rho_chunk, int32_t force_block);
rbe_status rbe_batch_get_tiles(rbe_batch b, int32_t* rho_k, int32_t* rho_chunk, int32_t* force_block);
/* Frequencies per lane of a rho tile: 1 (default) or 2.  With 2 each of the tile's rho_k lanes
 * holds two frequencies (the tile covers 2 rho_k), so that one staged particle record feeds two
 * (particle, frequency) pairs.  Kept by rbe_batch_set_tiles; reset to 1 by its all-zero
 * defaults; chosen with the other shapes by rbe_batch_autotune.  RBE_EINVAL for other values. */
rbe_status rbe_batch_set_rho_f(rbe_batch b, int32_t rho_f);
rbe_status rbe_batch_get_rho_f(rbe_batch b, int32_t* rho_f);

/* Evaluate items[0..n) (host array of descriptors, read during the call).  Asynchronous on the
 * batch's stream; validation errors (RBE_EINVAL) leave no side effects.  The work lists are
 * rebuilt (with a synchronisation of the stream) only when some item's N or a tile shape
 * changed.  Graph capture: evaluate the same items once outside capture first (RBE_ESTATE
 * otherwise); a captured evaluation reads the descriptors as they are at replay, so make no
 * other call on the batch between capture and replay.  Device errors (m = 0 after 2^20
 * redraws, non-finite values) are reported by rbe_batch_sync. */
rbe_status rbe_kspace_forces_virial_batched(rbe_batch b, const rbe_batch_item* items, int32_t n);

/* Times candidate tile shapes on these items (rho lanes x frequencies per lane x particles per
 * chunk, then particles per force tile; reps evaluations of each pass; with the persistent launch
 * on, the force tiles on reps whole evaluations) and keeps the fastest; the items' outputs are
 * overwritten.  *best_ms (may be NULL): mean time of one evaluation with
 * the chosen shapes.  Synchronous. */
rbe_status rbe_batch_autotune(rbe_batch b, const rbe_batch_item* items, int32_t n, int32_t reps, double* best_ms);

/* 1 (default): one persistent cooperative launch per evaluation; 0: one launch per pass, each of
 * a kernel compiled for that pass alone (fewer registers, more resident blocks; the same tile
 * bodies and results, bit for bit).  RBE_EINVAL for other values. */
rbe_status rbe_batch_set_persistent(rbe_batch b, int32_t enable);

/* Test of the failure path of the persistent launch (no counterpart in the paper): with
 * enable = 1 the grid barriers of later persistent evaluations wait for one block more than the
 * grid has, so every wait runs out after its one-second limit, the blocks leave the kernel, and
 * rbe_batch_sync reports RBE_ETIMEOUT (the outputs of that evaluation are incomplete); 0
 * restores normal operation, and the next evaluation is complete again.  RBE_EINVAL for other
 * values. */
rbe_status rbe_batch_test_barrier_timeout(rbe_batch b, int32_t enable);

/* Waits for the batch's stream and reports device-side errors of earlier evaluations. */
rbe_status rbe_batch_sync(rbe_batch b);
const char* rbe_batch_last_error(rbe_batch b);

/* ---------------------------------------------------------------------------------
 * Serving loop for independent NPT replicas (continuous batching on one GPU; no counterpart
 * in the paper, whose runs are single systems).  Requests queue on the host; a request is
 * admitted when a slot is free and its device memory fits the budget, and its state stays
 * resident in HBM until it finishes.  Each resident replica runs on its own non-blocking
 * stream and context, in chunks of chunk_steps NPT steps (rbe_npt_step), captured once per
 * replica as a CUDA graph when use_graphs != 0; chunks of different replicas run
 * concurrently, and requests are admitted while others run.  A replica's result does not
 * depend on what else is resident (no shared state; fixed-order reductions). */
typedef struct rbe_server_s* rbe_server;

typedef struct {
    double alpha;        /* Ewald splitting of every replica */
    int32_t P;           /* RBE batch size */
    int32_t precision;   /* rbe_precision */
    int32_t max_slots;   /* replicas resident at once, 1..4096 */
    int32_t chunk_steps; /* NPT steps per chunk, >= 1 */
    int64_t mem_budget;  /* device bytes the resident replicas may use; a replica of N particles
                            counts N*196 + 12*C + (P+1)*32768 + 4 MiB bytes (state, NPT scratch,
                            C = prod_t floor(2 l_t / rc) cells, tables), plus N*(4*cap + 20) with a
                            neighbour list (cap = 2 x the expected neighbours within rc + skin, + 64,
                            rounded up to 32), plus 128 (P + ptilde) + 16 reuse (P + ptilde) for the
                            frequency buffers (the reuse term when reuse > 1) */
    int32_t use_graphs;  /* 1: replay a captured graph per chunk; 0: launch the steps directly */
    int32_t batched;     /* 0: every replica runs its own chunks (its own stream and graph).  1: the
                            resident replicas advance in lockstep chunks; each step's k-space of all
                            of them is one persistent batched launch (rbe_batch, the tiles autotuned
                            on the group), their cell updates, drifts, real space and finishing
                            kernels run on their own streams around it, and a group that stays the
                            same for a second chunk is captured as one CUDA graph and replayed.
                            The batch runs its default tile shapes (1), or (2) the shapes
                            rbe_batch_autotune picks on the first group captured, kept for the
                            server's life.  FP32-phase only; requests with the exact sampler, no
                            pressure batch and no sample reuse, the k-space on.  Requests join and
                            leave at chunk boundaries.  A replica's result depends on its own data
                            and the tile shapes only, not on the other replicas of its group. */
} rbe_server_config;

typedef struct {
    int64_t N;
    const double* pos;     /* host N*3 (copied at submission) */
    const double* mom;     /* host N*3 */
    const double* charge;  /* host N */
    const double* mass;    /* host N */
    double box[3];
    double pV;             /* initial piston momentum */
    uint64_t seed;         /* Philox key of this replica (RBE batches and noise) */
    int32_t nsteps;        /* steps to run, >= 1 */
    int32_t pad;
    rbe_npt_params params;
    double pc[3];          /* initial cell momenta of barostats 2 and 3 (cell[12..14]) */
    int32_t sampler;       /* rbe_sampler of this replica's frequencies (rbe_set_sampler) */
    int32_t ptilde;        /* >= 0: a separate pressure batch (rbe_set_pressure_batch) */
    int32_t reuse;         /* samples drawn every `reuse` steps (rbe_set_sample_reuse, <= 1024); 0 or 1:
                              every step; excluded with the Metropolis--Hastings sampler */
    int32_t pad2;
} rbe_request;

rbe_status rbe_server_create(const rbe_server_config* cfg, rbe_server* out);
rbe_status rbe_server_destroy(rbe_server s);

/* Enqueue a request (inputs are copied, the caller may reuse its buffers); *id counts from 0.
 * RBE_ENOMEM if the request alone exceeds the memory budget. */
rbe_status rbe_server_submit(rbe_server s, const rbe_request* req, int64_t* id);

/* One round of the loop: observe finished chunks (non-blocking event queries), retire
 * finished requests (their results are copied to host memory), admit queued requests in
 * arrival order while a slot is free and the budget allows, and launch the next chunk of
 * every idle resident replica.  With wait != 0 it repeats until at least one chunk has
 * finished (or nothing is left).  Outputs (may be NULL): queued, resident, finished counts. */
rbe_status rbe_server_progress(rbe_server s, int32_t wait, int32_t* n_queued, int32_t* n_active, int64_t* n_done);

/* Cancel a request: a queued one leaves the queue at once; a resident one leaves its slot at
 * the end of its chunk in flight (observed by a later rbe_server_progress), and its slot serves
 * the next request.  A cancelled request counts as done; its result is RBE_ESTATE ("request
 * cancelled").  RBE_ESTATE for a request that has already finished, RBE_EINVAL for an unknown
 * id.  The other requests are unaffected. */
rbe_status rbe_server_cancel(rbe_server s, int64_t id);

/* Where a request stands: *state 0 queued, 1 resident, 2 finished, 3 failed, 4 cancelled; *error
 * the failure's status (RBE_OK unless 3 or 4).  Either pointer may be NULL.  A resident
 * replica whose device status word latched an error (non-finite values, a box outside the
 * range rbe_npt_init prepared, a full neighbour list, ...) is evicted at the end of the chunk
 * that raised it: the server reads every replica's status word after each chunk, and that
 * replica fails with the error while the others run on. */
rbe_status rbe_server_request_state(rbe_server s, int64_t id, int32_t* state, rbe_status* error);

/* Final state of a finished request into host memory (any pointer may be NULL): pos, mom
 * N*3 and the cell block (RBE_CELL_DOUBLES).  RBE_ESTATE while it runs or after it was
 * cancelled; the failure's status (with its message in rbe_server_last_error) for a request
 * that failed. */
rbe_status rbe_server_result(rbe_server s, int64_t id, double* pos, double* mom, double* cell);

/* Per-chunk latencies in seconds (launch to observed completion), up to `capacity` of them;
 * the number of chunks and steps finished; the span from the first admission to the last
 * retirement. */
rbe_status rbe_server_stats(rbe_server s, double* chunk_latency, int64_t capacity, int64_t* n_chunks,
                            int64_t* steps_done, double* span_seconds);

/* Message for the server's last failure. */
const char* rbe_server_last_error(rbe_server s);

/* Static description of a status code. */
const char* rbe_status_string(rbe_status status);

/* Message for the last non-OK status returned on ctx (or by rbe_create when ctx is NULL). */
const char* rbe_last_error(rbe_ctx ctx);

/* Library version as major*10000 + minor*100 + patch. */
int32_t rbe_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RBE_H */
