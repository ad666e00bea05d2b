/*
 * Parameters of the oracle's Langevin NPT steps (npt_oracle.c; the rigid-water step of
 * water_oracle.c uses the isotropic fields) -- TEST INFRASTRUCTURE ONLY (conventions and who may
 * load it: rbe_oracle.c).  Mirrored by NptParams in oracle/__init__.py.
 */
#ifndef ORC_NPT_PARAMS_H
#define ORC_NPT_PARAMS_H
#include <stdint.h>

typedef struct {
    double dt;        /* ps */
    double kT;        /* kJ/mol */
    double P_ext;     /* kJ/mol/A^3 */
    double gamma;     /* particle friction, 1/ps */
    double gamma_V;   /* cell friction, 1/ps */
    double M_V;       /* piston mass, kJ/mol ps^2 / A^6 */
    double alpha;     /* Ewald splitting, A^-2 */
    double rc;        /* real-space cutoff, A */
    double qqr2e;     /* Coulomb constant, kJ/mol A / e^2 */
    double lj_sigma;  /* A */
    double lj_eps;    /* kJ/mol (0: no Lennard-Jones) */
    double max_disp;  /* cap on the peculiar |dr| per step, half per R/2 sub-step, A (0: none) */
    int32_t P;        /* RBE batch size */
    int32_t kspace;   /* 1: RBE k-space forces and virial */
    int32_t real;     /* 1: erfc Coulomb + LJ real space */
    int32_t noise;    /* 1: Langevin noise in O and O^p */
    int32_t barostat; /* 1: the cell moves (V^p, V, O^p); 0: V fixed, p_V = 0;
                         2: rectangular cell, anisotropic; 3: semi-isotropic (orc_npt_step_rect) */
    int32_t pad;
    uint64_t seed;
    double M_cell[3]; /* barostat 2: masses of l_x, l_y, l_z (kJ/mol ps^2/A^2);
                         barostat 3: M_A (kJ/mol ps^2/A^4) in [0], M_L (kJ/mol ps^2/A^2) in [2] */
    double gamma0;    /* barostat 3: surface tension times the number of surfaces, kJ/mol/A^2 */
    int32_t sampler;  /* frequencies: 0 exact, 1 offline, 2 Metropolis--Hastings (sampler_oracle.c) */
    int32_t pad2;
    int32_t* chain;   /* sampler 2: the chain state, (P + Ptilde) x 3 (in/out; rows of zeros start exact) */
    int32_t Ptilde;   /* > 0: a separate pressure batch (Eq. (apppress)) of Ptilde frequencies for the
                         virial and the k-space energy, slots [P, P + Ptilde) of the same draw */
    int32_t reuse;    /* > 1: samples drawn every `reuse` steps (Sec. 4.3): at a step s with
                         s mod reuse = 0, reuse batches of P + Ptilde slots from the box of step s
                         into reuse_m; step s + i evaluates batch i with its own box's k and S */
    int32_t* reuse_m; /* reuse x (P + Ptilde) x 3 (kept between steps) */
} orc_npt_params;

#endif
