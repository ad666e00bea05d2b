/*
 * Oracle for the isotropic Langevin NPT step driven by the RBE forces -- TEST
 * INFRASTRUCTURE ONLY (see rbe_oracle.c for the conventions and who may load it).
 *
 * Equations of motion (Sec. 3.2, the isotropic Langevin equations):
 *   dr/dt = p/m + (dV/dt)/(3V) r,   dp/dt = F - (dV/dt)/(3V) p - gamma p + sqrt(2 kT m gamma) xi,
 *   dV/dt = p_V / M,                dp_V/dt = P_ins - P - gamma_V p_V + sqrt(2 kT gamma_V M) xi_V,
 * discretised by the symmetric splitting of Sec. 3.3:
 *   V^p/2, R^p/2, V/2, R/2, O^p, O, R/2, V/2, [forces and P_ins], R^p/2, V^p/2,
 * where R and R^p are solved exactly with eps = p_V / (3 M V) frozen over the sub-step,
 * and O, O^p are the exact Ornstein--Uhlenbeck updates p <- e^{-g t} p + sqrt(kT m (1 - e^{-2 g t})) R.
 * The forces and the pressure are evaluated after the second V/2 (Sec. 3.3, last paragraph).
 * P_ins = (sum p^2/m + W_k + W_r) / (3V) (Sec. 4.1 Eq. (pressurecubic); the real-space virial
 * taken as -3V dU_2/dV).
 *
 * Units: A, ps, g/mol, kJ/mol, e.  Forces in kJ/mol/A; dp/dt = 100 F (g/mol A/ps^2 per
 * kJ/mol/A); kinetic energy sum p^2/(2m) / 100 in kJ/mol; pressure in kJ/mol/A^3;
 * p_V in kJ/mol ps / A^3 and M in kJ/mol ps^2 / A^6.  The box scales isotropically
 * (all three lengths by (V'/V)^(1/3)).
 *
 * Random numbers: Philox-4x32-10 with key (seed_lo, seed_hi); particle noise uses the
 * counter (i, 0, step_lo, (1 << 24) | step_hi24), the cell noise (0, 0, step_lo,
 * (2 << 24) | step_hi24); each 32-bit word w gives u = (w + 0.5) 2^-32, and Box--Muller
 * turns (u0, u1), (u2, u3) into four standard normals, of which a particle uses three.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { NPT_OK = 0, NPT_EINVAL = 1, NPT_ENOMEM = 2 };

#define FCONV 100.0 /* kJ/mol/A per g/mol -> A/ps^2 */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
int orc_sample_k(const double box[3], double alpha, int32_t P, uint64_t seed, uint64_t step,
                 int32_t* m_out, double* S_out);
int orc_sample_k_offline(const double box[3], double alpha, int32_t P, uint64_t seed, uint64_t step,
                         int32_t* m_out, double* S_out);
int orc_sample_k_mh(const double box[3], double alpha, int32_t P, uint64_t seed, uint64_t step, int32_t* state,
                    double* S_out);
int orc_rbe_kspace(int64_t N, const double* pos, const double* q, const double box[3], double alpha,
                   int32_t P, const int32_t* m, const double* wl, double* F, double W[9], double E[2],
                   double* rho);

#include "npt_params.h"

/* ------------------------------------------------------------------------------ */
/* Standard normals from one Philox call (Box--Muller). */
void orc_npt_normals(uint64_t seed, uint32_t stream, uint64_t step, uint32_t index, double z[4])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {index, 0u, (uint32_t)step, (stream << 24) | (uint32_t)((step >> 32) & 0xFFFFFFu)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    double u[4];
    for (int j = 0; j < 4; ++j) u[j] = ((double)w[j] + 0.5) * 0x1.0p-32;
    for (int j = 0; j < 2; ++j) {
        double rad = sqrt(-2.0 * log(u[2 * j]));
        z[2 * j] = rad * cos(2.0 * M_PI * u[2 * j + 1]);
        z[2 * j + 1] = rad * sin(2.0 * M_PI * u[2 * j + 1]);
    }
}

/* ------------------------------------------------------------------------------ */
/* Real-space forces with the nearest image inside rc (Sec. 4.1 Eqs. (U2), (force); Sec. 4.2):
 *   U = sum_{i<j, r<rc} [qqr2e q_i q_j erfc(sqrt(a) r)/r + 4 eps ((s/r)^12 - (s/r)^6)]
 * d = r_j - r_i (nearest image); the force on j is f d with f = -(dU/dr)/r, on i its negative;
 * W = sum_{i<j} f d (x) d.  E[0] = Coulomb part, E[1] = Lennard-Jones part. */
int orc_pair_real(int64_t N, const double* pos, const double* q, const double box[3], double alpha, double rc,
                  double qqr2e, double lj_sigma, double lj_eps, double* F, double W[9], double E[2])
{
    if (N < 0 || !(rc > 0.0)) return NPT_EINVAL;
    for (int t = 0; t < 3; ++t)
        if (!(box[t] > 0.0) || rc > 0.5 * box[t]) return NPT_EINVAL;
    for (int64_t i = 0; i < 3 * N; ++i) F[i] = 0.0;
    for (int j = 0; j < 9; ++j) W[j] = 0.0;
    E[0] = 0.0;
    E[1] = 0.0;
    double sa = sqrt(alpha);
    for (int64_t i = 0; i < N; ++i) {
        for (int64_t j = i + 1; j < N; ++j) {
            double d[3];
            for (int t = 0; t < 3; ++t) {
                double x = pos[3 * j + t] - pos[3 * i + t];
                d[t] = x - box[t] * nearbyint(x / box[t]);
            }
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < rc * rc)) continue;
            double r = sqrt(r2);
            double qq = qqr2e * q[i] * q[j];
            double ec = erfc(sa * r);
            double f = qq * (ec / r2 + 2.0 * sa * exp(-alpha * r2) / (sqrt(M_PI) * r)) / r;
            E[0] += qq * ec / r;
            if (lj_eps != 0.0) {
                double sr2 = lj_sigma * lj_sigma / r2;
                double sr6 = sr2 * sr2 * sr2;
                E[1] += 4.0 * lj_eps * (sr6 * sr6 - sr6);
                f += 24.0 * lj_eps * (2.0 * sr6 * sr6 - sr6) / r2;
            }
            for (int t = 0; t < 3; ++t) {
                F[3 * j + t] += f * d[t];
                F[3 * i + t] -= f * d[t];
            }
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) W[3 * a + c] += f * d[a] * d[c];
        }
    }
    return NPT_OK;
}

/* Forces (kJ/mol/A), the trace of the virial (kJ/mol) and, if Wd is given, its diagonal, at
 * the current state: RBE k-space with the batch of `step` (Sec. 4.2 Eqs. (appforce),
 * (apppress)) times qqr2e, plus the real space.  Energies: E[0] k-space (incl. self),
 * E[1] real Coulomb, E[2] Lennard-Jones. */
static int npt_forces_parts(int64_t N, const double* r, const double* q, const double L[3], uint64_t step,
                            const orc_npt_params* prm, double* F, double* Wtr, double* Wd, double E[3])
{
    double* Fk = (double*)calloc((size_t)(3 * N + 3), sizeof(double));
    if (!Fk) return NPT_ENOMEM;
    for (int64_t i = 0; i < 3 * N; ++i) F[i] = 0.0;
    double W = 0.0;
    if (Wd) Wd[0] = Wd[1] = Wd[2] = 0.0;
    E[0] = E[1] = E[2] = 0.0;
    int st = NPT_OK;
    if (prm->kspace) {
        /* force batch: slots [0, P), weights S/P (Eq. (appforce)); pressure batch: slots
         * [P, P + Ptilde), weights S/Ptilde (Eq. (apppress)), or the force batch when Ptilde = 0 */
        const int32_t Pt = prm->Ptilde > 0 ? prm->Ptilde : 0;
        const int32_t Ptot = prm->P + Pt;
        int32_t* m = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(Ptot > 0 ? Ptot : 1));
        double* wl = (double*)malloc(sizeof(double) * (size_t)(Ptot > 0 ? Ptot : 1));
        double* Fp = Pt > 0 ? (double*)calloc((size_t)(3 * N + 3), sizeof(double)) : NULL;
        if (!m || !wl || (Pt > 0 && !Fp)) {
            free(m); free(wl); free(Fp); free(Fk);
            return NPT_ENOMEM;
        }
        double S = 0.0, Wk[9], Ek[2];
        if (prm->reuse > 1 && prm->sampler != 2) {
            const int32_t i = (int32_t)(step % (uint64_t)prm->reuse);
            if (!prm->reuse_m) {
                st = NPT_EINVAL;
            } else if (i == 0) {
                /* draw every batch from this step's box (batch 0 is the ordinary draw) */
                int32_t Pall = prm->reuse * Ptot;
                st = prm->sampler == 1 ? orc_sample_k_offline(L, prm->alpha, Pall, prm->seed, step, prm->reuse_m, &S)
                                       : orc_sample_k(L, prm->alpha, Pall, prm->seed, step, prm->reuse_m, &S);
            }
            /* S of the current box (the weights), batch i of the kept draws */
            if (st == NPT_OK) st = orc_sample_k(L, prm->alpha, 0, prm->seed, step, NULL, &S);
            for (int32_t j = 0; st == NPT_OK && j < 3 * Ptot; ++j) m[j] = prm->reuse_m[3 * (size_t)i * Ptot + j];
        } else if (prm->reuse > 1) {
            st = NPT_EINVAL; /* reuse and the Metropolis--Hastings chain exclude each other */
        } else if (prm->sampler == 1) {
            st = orc_sample_k_offline(L, prm->alpha, Ptot, prm->seed, step, m, &S);
        } else if (prm->sampler == 2) {
            if (!prm->chain) {
                st = NPT_EINVAL;
            } else {
                st = orc_sample_k_mh(L, prm->alpha, Ptot, prm->seed, step, prm->chain, &S);
                for (int32_t j = 0; st == NPT_OK && j < 3 * Ptot; ++j) m[j] = prm->chain[j];
            }
        } else {
            st = orc_sample_k(L, prm->alpha, Ptot, prm->seed, step, m, &S);
        }
        if (st == NPT_OK) {
            for (int32_t l = 0; l < prm->P; ++l) wl[l] = S / (double)prm->P;
            for (int32_t l = prm->P; l < Ptot; ++l) wl[l] = S / (double)Pt;
            st = orc_rbe_kspace(N, r, q, L, prm->alpha, prm->P, m, wl, Fk, Wk, Ek, NULL);
        }
        if (st == NPT_OK && Pt > 0)
            st = orc_rbe_kspace(N, r, q, L, prm->alpha, Pt, m + 3 * prm->P, wl + prm->P, Fp, Wk, Ek, NULL);
        if (st == NPT_OK) {
            for (int64_t i = 0; i < 3 * N; ++i) F[i] += prm->qqr2e * Fk[i];
            W += prm->qqr2e * (Wk[0] + Wk[4] + Wk[8]);
            if (Wd)
                for (int t = 0; t < 3; ++t) Wd[t] = prm->qqr2e * Wk[4 * t];
            E[0] = prm->qqr2e * (Ek[0] + Ek[1]);
        }
        free(m);
        free(wl);
        free(Fp);
    }
    if (st == NPT_OK && prm->real) {
        double Wr[9], Er[2];
        st = orc_pair_real(N, r, q, L, prm->alpha, prm->rc, prm->qqr2e, prm->lj_sigma, prm->lj_eps, Fk, Wr, Er);
        if (st == NPT_OK) {
            for (int64_t i = 0; i < 3 * N; ++i) F[i] += Fk[i];
            W += Wr[0] + Wr[4] + Wr[8];
            if (Wd)
                for (int t = 0; t < 3; ++t) Wd[t] += Wr[4 * t];
            E[1] = Er[0];
            E[2] = Er[1];
        }
    }
    free(Fk);
    *Wtr = W;
    return st;
}

int orc_npt_forces(int64_t N, const double* r, const double* q, const double L[3], uint64_t step,
                   const orc_npt_params* prm, double* F, double* Wtr, double E[3])
{
    return npt_forces_parts(N, r, q, L, step, prm, F, Wtr, NULL, E);
}

/* The same with the diagonal W_jj of the virial (k-space and real space) in Wd. */
int orc_npt_forces_diag(int64_t N, const double* r, const double* q, const double L[3], uint64_t step,
                        const orc_npt_params* prm, double* F, double Wd[3], double E[3])
{
    double Wtr;
    return npt_forces_parts(N, r, q, L, step, prm, F, &Wtr, Wd, E);
}

/* ------------------------------------------------------------------------------ */
/* Exact sub-step solutions with eps frozen (Sec. 3.3: the R and R^p flows).
 * x(t) = x e^{s eps t} + v (e^{s eps t} - 1) / (s eps) for dx/dt = v + s eps x (s = +1 for R,
 * s = -1 for R^p); the ratio is expanded when |eps t| is small. */
static double expm1_over(double x, double t)
{
    /* (e^{x} - 1) / x * t  with x = eps t, written as t * (1 + x/2 + x^2/6 + x^3/24) for tiny x */
    if (fabs(x) < 1e-8) return t * (1.0 + x * (0.5 + x * (1.0 / 6.0 + x / 24.0)));
    return t * expm1(x) / x;
}

static double kinetic2(int64_t N, const double* p, const double* m)
{
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i)
        s += (p[3 * i] * p[3 * i] + p[3 * i + 1] * p[3 * i + 1] + p[3 * i + 2] * p[3 * i + 2]) / m[i];
    return s / FCONV; /* = 2 K in kJ/mol */
}

static void scale_box(double L[3], double Vnew)
{
    double V = L[0] * L[1] * L[2];
    double f = cbrt(Vnew / V);
    for (int t = 0; t < 3; ++t) L[t] *= f;
}

/* V^p/2 */
static void half_kick_cell(double* pV, double Pins, const orc_npt_params* prm)
{
    if (prm->barostat) *pV += 0.5 * prm->dt * (Pins - prm->P_ext);
}

/* R^p/2: p <- p e^{-eps h} + 100 F (1 - e^{-eps h}) / eps */
static void half_kick_particles(int64_t N, double* p, const double* F, double eps, double h)
{
    double a = exp(-eps * h);
    double b = expm1_over(-eps * h, h); /* (e^{-eps h} - 1) / (-eps) */
    for (int64_t i = 0; i < 3 * N; ++i) p[i] = p[i] * a + FCONV * F[i] * b;
}

/* The optional cap on the displacement of one R/2 sub-step applies to its peculiar part
 * (p/m) (e^{eps h} - 1)/eps only: the affine part r (e^{eps h} - 1) is the cell's dilation,
 * which every particle follows (capping it would hold back the particles far from the
 * origin and distort the box). */
static void cap_peculiar(double d[3], double cap)
{
    if (cap > 0.0) {
        double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (len > cap)
            for (int t = 0; t < 3; ++t) d[t] *= cap / len;
    }
}

/* R/2: r <- r e^{eps h} + (p/m) (e^{eps h} - 1) / eps, with the optional cap */
static void half_drift(int64_t N, double* r, const double* p, const double* m, double eps, double h, double cap)
{
    double a = exp(eps * h);
    double b = expm1_over(eps * h, h);
    for (int64_t i = 0; i < N; ++i) {
        double d[3];
        for (int t = 0; t < 3; ++t) d[t] = (p[3 * i + t] / m[i]) * b;
        cap_peculiar(d, cap);
        for (int t = 0; t < 3; ++t) r[3 * i + t] += r[3 * i + t] * (a - 1.0) + d[t];
    }
}

/* One step.  State in/out: r, p, F (forces at r), L (box), pV, Wtr (virial trace at r).
 * F and Wtr must hold the values at the input state (orc_npt_forces at `step` - 1 or an
 * initial evaluation); on return they hold the values at the new state, evaluated with the
 * RBE batch of `step`. */
int orc_npt_step(int64_t N, double* r, double* p, double* F, const double* q, const double* m, double L[3],
                 double* pV, double* Wtr, uint64_t step, const orc_npt_params* prm, double E[3])
{
    if (prm->barostat < 0 || prm->barostat > 1) return NPT_EINVAL; /* rectangular cells: orc_npt_step_rect */
    const double h = 0.5 * prm->dt;
    double V = L[0] * L[1] * L[2];
    /* V^p/2 with the pressure of the current state */
    double Pins = (kinetic2(N, p, m) + *Wtr) / (3.0 * V);
    half_kick_cell(pV, Pins, prm);
    double eps = prm->barostat ? *pV / (3.0 * prm->M_V * V) : 0.0;
    /* R^p/2 */
    half_kick_particles(N, p, F, eps, h);
    /* V/2 */
    if (prm->barostat) {
        double Vn = V + h * (*pV) / prm->M_V;
        scale_box(L, Vn);
        V = L[0] * L[1] * L[2];
    }
    eps = prm->barostat ? *pV / (3.0 * prm->M_V * V) : 0.0;
    /* R/2 */
    half_drift(N, r, p, m, eps, h, 0.5 * prm->max_disp);
    /* O^p */
    if (prm->barostat) {
        double g = exp(-prm->gamma_V * prm->dt);
        *pV *= g;
        if (prm->noise) {
            double z[4];
            orc_npt_normals(prm->seed, 2u, step, 0u, z);
            *pV += sqrt(prm->kT * prm->M_V * (1.0 - g * g)) * z[0];
        }
    }
    /* O */
    {
        double g = exp(-prm->gamma * prm->dt);
        for (int64_t i = 0; i < N; ++i) {
            double z[4] = {0.0, 0.0, 0.0, 0.0};
            if (prm->noise) orc_npt_normals(prm->seed, 1u, step, (uint32_t)i, z);
            double s = sqrt(prm->kT * FCONV * m[i] * (1.0 - g * g));
            for (int t = 0; t < 3; ++t) p[3 * i + t] = p[3 * i + t] * g + s * z[t];
        }
    }
    eps = prm->barostat ? *pV / (3.0 * prm->M_V * V) : 0.0;
    /* R/2 */
    half_drift(N, r, p, m, eps, h, 0.5 * prm->max_disp);
    /* V/2 */
    if (prm->barostat) {
        double Vn = V + h * (*pV) / prm->M_V;
        scale_box(L, Vn);
        V = L[0] * L[1] * L[2];
    }
    /* wrap into the new box */
    for (int64_t i = 0; i < N; ++i)
        for (int t = 0; t < 3; ++t) r[3 * i + t] -= L[t] * floor(r[3 * i + t] / L[t]);
    /* forces and virial at the new state */
    int st = orc_npt_forces(N, r, q, L, step, prm, F, Wtr, E);
    if (st != NPT_OK) return st;
    eps = prm->barostat ? *pV / (3.0 * prm->M_V * V) : 0.0;
    /* R^p/2 */
    half_kick_particles(N, p, F, eps, h);
    /* V^p/2 with the momenta after R^p/2 */
    Pins = (kinetic2(N, p, m) + *Wtr) / (3.0 * V);
    half_kick_cell(pV, Pins, prm);
    return NPT_OK;
}

/* n steps from step0; records V, P_ins (after each step) and the extended energy
 * K + U + P V + p_V^2/(2M) into the optional arrays. */
int orc_npt_run(int64_t N, double* r, double* p, double* F, const double* q, const double* m, double L[3],
                double* pV, double* Wtr, uint64_t step0, int32_t nsteps, const orc_npt_params* prm,
                double* V_out, double* Pins_out, double* H_out)
{
    for (int32_t s = 0; s < nsteps; ++s) {
        double E[3];
        int st = orc_npt_step(N, r, p, F, q, m, L, pV, Wtr, step0 + (uint64_t)s, prm, E);
        if (st != NPT_OK) return st;
        double V = L[0] * L[1] * L[2];
        double K2 = kinetic2(N, p, m);
        if (V_out) V_out[s] = V;
        if (Pins_out) Pins_out[s] = (K2 + *Wtr) / (3.0 * V);
        if (H_out)
            H_out[s] = 0.5 * K2 + E[0] + E[1] + E[2] + prm->P_ext * V +
                       (prm->barostat ? (*pV) * (*pV) / (2.0 * prm->M_V) : 0.0);
    }
    return NPT_OK;
}

/* ------------------------------------------------------------------------------ */
/* Rectangular cell with per-axis fluctuation (appendix: the rectangular cell with
 * anisotropic fluctuation, and the semi-isotropic constant surface-tension case).
 *
 * Anisotropic (barostat 2): h = diag(l_1, l_2, l_3), V = l_1 l_2 l_3,
 *   dr_j/dt = p_j/m + eps_j r_j,   dp_j/dt = F_j - eps_j p_j - gamma p_j + noise,   eps_j = (dl_j/dt)/l_j,
 *   dl_j/dt = pc_j / M_j,          dpc_j/dt = V ((P_ins)_jj - P) / l_j - gamma_V pc_j + sqrt(2 kT gamma_V M_j) xi_j,
 * with (P_ins)_jj = (sum_i p_ij^2/m_i + W_jj) / V (the diagonal pressure of the rectangular
 * cell).  Extended energy K + U + P V + sum_j pc_j^2 / (2 M_j).
 *
 * Semi-isotropic (barostat 3): h = diag(sqrt(A), sqrt(A), L) (a square cross-section, l_x = l_y),
 *   eps_x = eps_y = (dA/dt)/(2A), eps_z = (dL/dt)/L,
 *   dA/dt = p^A / M_A,   dp^A/dt = L (P_A - P) - gamma_V p^A + sqrt(2 kT gamma_V M_A) xi_A,
 *   dL/dt = p^L / M_L,   dp^L/dt = A ((P_ins)_zz - P) - gamma_V p^L + sqrt(2 kT gamma_V M_L) xi_L,
 * with P_A = ((P_ins)_xx + (P_ins)_yy)/2 + gamma0 / L.  Extended energy
 * K + U + P A L - gamma0 A + (p^A)^2/(2 M_A) + (p^L)^2/(2 M_L).  One friction gamma_V serves
 * both cell variables.
 *
 * Cell momenta pc[3]: anisotropic {pc_x, pc_y, pc_z}; semi-isotropic {p^A, 0, p^L}.  The
 * splitting is the one of the isotropic step (Sec. 3.3) with the strain rate per axis:
 *   V^p/2, R^p/2, V/2, R/2, O^p, O, R/2, V/2, [forces, W_jj], R^p/2, V^p/2,
 * R and R^p solved exactly per axis with eps_j frozen; V/2 moves l_j (or A and L) linearly
 * with pc frozen.  O^p draws the cell normals z[0..3] from the cell counter (stream 2) and
 * gives slot j the normal z[j]. */
static int rect_check(const double L[3], const orc_npt_params* prm)
{
    if (prm->barostat == 2) {
        for (int j = 0; j < 3; ++j)
            if (!(prm->M_cell[j] > 0.0)) return NPT_EINVAL;
        return NPT_OK;
    }
    if (prm->barostat == 3) {
        if (!(prm->M_cell[0] > 0.0) || !(prm->M_cell[2] > 0.0) || L[0] != L[1]) return NPT_EINVAL;
        return NPT_OK;
    }
    return NPT_EINVAL;
}

/* eps_j = (dl_j/dt)/l_j for the current cell momenta and box */
static void rect_eps(const double L[3], const double pc[3], const orc_npt_params* prm, double eps[3])
{
    if (prm->barostat == 2) {
        for (int j = 0; j < 3; ++j) eps[j] = pc[j] / (prm->M_cell[j] * L[j]);
    } else {
        double A = L[0] * L[1];
        eps[0] = eps[1] = pc[0] / (2.0 * prm->M_cell[0] * A);
        eps[2] = pc[2] / (prm->M_cell[2] * L[2]);
    }
}

static void kinetic2_axes(int64_t N, const double* p, const double* m, double K2[3])
{
    for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int64_t i = 0; i < N; ++i) s += p[3 * i + j] * p[3 * i + j] / m[i];
        K2[j] = s / FCONV; /* sum_i p_ij^2 / m_i in kJ/mol */
    }
}

/* V^p/2: the cell momenta take half a step of their force -dH/d(cell variable) */
static void rect_kick_cell(double pc[3], const double L[3], const double K2[3], const double Wd[3],
                           const orc_npt_params* prm)
{
    const double h = 0.5 * prm->dt;
    if (prm->barostat == 2) {
        double V = L[0] * L[1] * L[2];
        for (int j = 0; j < 3; ++j) pc[j] += h * ((K2[j] + Wd[j] - prm->P_ext * V) / L[j]);
    } else {
        double A = L[0] * L[1];
        /* L (P_A - P) = (2K_x + W_xx + 2K_y + W_yy) / (2A) - P L + gamma0 */
        pc[0] += h * ((K2[0] + Wd[0] + K2[1] + Wd[1]) / (2.0 * A) - prm->P_ext * L[2] + prm->gamma0);
        /* A ((P_ins)_zz - P) = (2K_z + W_zz) / L - P A */
        pc[2] += h * ((K2[2] + Wd[2]) / L[2] - prm->P_ext * A);
    }
}

/* V/2: the cell variables move with their momenta frozen */
static void rect_move_cell(double L[3], const double pc[3], const orc_npt_params* prm)
{
    const double h = 0.5 * prm->dt;
    if (prm->barostat == 2) {
        for (int j = 0; j < 3; ++j) L[j] += h * pc[j] / prm->M_cell[j];
    } else {
        double A = L[0] * L[1] + h * pc[0] / prm->M_cell[0];
        L[0] = L[1] = sqrt(A);
        L[2] += h * pc[2] / prm->M_cell[2];
    }
}

/* R^p/2 per axis: p_j <- p_j e^{-eps_j h} + 100 F_j (1 - e^{-eps_j h}) / eps_j */
static void half_kick_particles_axes(int64_t N, double* p, const double* F, const double eps[3], double h)
{
    double a[3], b[3];
    for (int j = 0; j < 3; ++j) {
        a[j] = exp(-eps[j] * h);
        b[j] = expm1_over(-eps[j] * h, h);
    }
    for (int64_t i = 0; i < N; ++i)
        for (int j = 0; j < 3; ++j) p[3 * i + j] = p[3 * i + j] * a[j] + FCONV * F[3 * i + j] * b[j];
}

/* R/2 per axis: r_j <- r_j e^{eps_j h} + (p_j/m) (e^{eps_j h} - 1) / eps_j, with the cap on
 * the peculiar part */
static void half_drift_axes(int64_t N, double* r, const double* p, const double* m, const double eps[3], double h,
                            double cap)
{
    double a[3], b[3];
    for (int j = 0; j < 3; ++j) {
        a[j] = exp(eps[j] * h);
        b[j] = expm1_over(eps[j] * h, h);
    }
    for (int64_t i = 0; i < N; ++i) {
        double d[3];
        for (int j = 0; j < 3; ++j) d[j] = (p[3 * i + j] / m[i]) * b[j];
        cap_peculiar(d, cap);
        for (int j = 0; j < 3; ++j) r[3 * i + j] += r[3 * i + j] * (a[j] - 1.0) + d[j];
    }
}

/* One step of the rectangular cell.  State in/out: r, p, F (forces at r), L, pc, Wd (virial
 * diagonal at r).  F and Wd must hold the values at the input state (orc_npt_forces_diag);
 * on return they hold those of the new state, with the RBE batch of `step`. */
int orc_npt_step_rect(int64_t N, double* r, double* p, double* F, const double* q, const double* m, double L[3],
                      double pc[3], double Wd[3], uint64_t step, const orc_npt_params* prm, double E[3])
{
    int st = rect_check(L, prm);
    if (st != NPT_OK) return st;
    const double h = 0.5 * prm->dt;
    double K2[3], eps[3];
    /* V^p/2 with the pressure of the current state */
    kinetic2_axes(N, p, m, K2);
    rect_kick_cell(pc, L, K2, Wd, prm);
    /* R^p/2 */
    rect_eps(L, pc, prm, eps);
    half_kick_particles_axes(N, p, F, eps, h);
    /* V/2 */
    rect_move_cell(L, pc, prm);
    /* R/2 */
    rect_eps(L, pc, prm, eps);
    half_drift_axes(N, r, p, m, eps, h, 0.5 * prm->max_disp);
    /* O^p */
    {
        double g = exp(-prm->gamma_V * prm->dt);
        double z[4] = {0.0, 0.0, 0.0, 0.0};
        if (prm->noise) orc_npt_normals(prm->seed, 2u, step, 0u, z);
        for (int j = 0; j < 3; ++j) {
            if (prm->barostat == 3 && j == 1) continue;
            pc[j] *= g;
            if (prm->noise) pc[j] += sqrt(prm->kT * prm->M_cell[j] * (1.0 - g * g)) * z[j];
        }
    }
    /* O */
    {
        double g = exp(-prm->gamma * prm->dt);
        for (int64_t i = 0; i < N; ++i) {
            double z[4] = {0.0, 0.0, 0.0, 0.0};
            if (prm->noise) orc_npt_normals(prm->seed, 1u, step, (uint32_t)i, z);
            double s = sqrt(prm->kT * FCONV * m[i] * (1.0 - g * g));
            for (int t = 0; t < 3; ++t) p[3 * i + t] = p[3 * i + t] * g + s * z[t];
        }
    }
    /* R/2 */
    rect_eps(L, pc, prm, eps);
    half_drift_axes(N, r, p, m, eps, h, 0.5 * prm->max_disp);
    /* V/2 */
    rect_move_cell(L, pc, prm);
    /* wrap into the new box */
    for (int64_t i = 0; i < N; ++i)
        for (int t = 0; t < 3; ++t) r[3 * i + t] -= L[t] * floor(r[3 * i + t] / L[t]);
    /* forces and virial diagonal at the new state */
    st = orc_npt_forces_diag(N, r, q, L, step, prm, F, Wd, E);
    if (st != NPT_OK) return st;
    /* R^p/2 */
    rect_eps(L, pc, prm, eps);
    half_kick_particles_axes(N, p, F, eps, h);
    /* V^p/2 with the momenta after R^p/2 */
    kinetic2_axes(N, p, m, K2);
    rect_kick_cell(pc, L, K2, Wd, prm);
    return NPT_OK;
}

/* n steps from step0; records per step the box (L_out, 3 per step), the diagonal pressure
 * (P_out, 3 per step) and the extended energy (H_out), each optional. */
int orc_npt_run_rect(int64_t N, double* r, double* p, double* F, const double* q, const double* m, double L[3],
                     double pc[3], double Wd[3], uint64_t step0, int32_t nsteps, const orc_npt_params* prm,
                     double* L_out, double* P_out, double* H_out)
{
    for (int32_t s = 0; s < nsteps; ++s) {
        double E[3], K2[3];
        int st = orc_npt_step_rect(N, r, p, F, q, m, L, pc, Wd, step0 + (uint64_t)s, prm, E);
        if (st != NPT_OK) return st;
        double V = L[0] * L[1] * L[2];
        kinetic2_axes(N, p, m, K2);
        for (int j = 0; j < 3; ++j) {
            if (L_out) L_out[3 * s + j] = L[j];
            if (P_out) P_out[3 * s + j] = (K2[j] + Wd[j]) / V;
        }
        if (H_out) {
            double H = 0.5 * (K2[0] + K2[1] + K2[2]) + E[0] + E[1] + E[2] + prm->P_ext * V;
            if (prm->barostat == 2) {
                for (int j = 0; j < 3; ++j) H += pc[j] * pc[j] / (2.0 * prm->M_cell[j]);
            } else {
                H += -prm->gamma0 * L[0] * L[1] + pc[0] * pc[0] / (2.0 * prm->M_cell[0]) +
                     pc[2] * pc[2] / (2.0 * prm->M_cell[2]);
            }
            H_out[s] = H;
        }
    }
    return NPT_OK;
}
