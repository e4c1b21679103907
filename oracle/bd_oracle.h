/*
 * Plain CPU FP64 oracle for replica-averaged Brownian dynamics
 * (Kania, Nguyen, Oztekin & Webb, "Replica-Averaging", arXiv 2206.05851).
 *
 * TEST INFRASTRUCTURE ONLY. This code is the slow, obviously-correct
 * reference the CUDA path is checked against. Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it; the product
 * library never links, includes or calls it, and it shares no code with it.
 *
 * Units: length l_H = sqrt(kT/H0), time lambda_H = zeta/(4 H0), kT = 1, so the
 * free-draining diffusivity kT/zeta of Eq. 2 is D = 1/4 and Eq. 1 becomes
 *   r_i <- r_i + [kappa . r_i + D (F_i - F_{i-1})] dt + sqrt(2 D dt) xi_i .
 */
#ifndef BD_ORACLE_H
#define BD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_SPRING_HOOKE = 0, ORA_SPRING_FENE = 1, ORA_SPRING_HARMONIC = 2, ORA_SPRING_VWF = 3 };
enum { ORA_FLOW_NONE = 0, ORA_FLOW_SHEAR = 1, ORA_FLOW_UNIAXIAL = 2, ORA_FLOW_PLANAR = 3 };
enum { ORA_ISF = 0, ORA_TSF = 1, ORA_RSF = 2 };          /* criterion index q */
enum { ORA_STREAM_BD = 0, ORA_STREAM_EXP1 = 1 };         /* Philox stream ids */

typedef struct {
    int32_t n_beads, n_replicas, spring, flow;
    double H, b, rate;     /* stiffness / H0, FENE b, flow rate in 1/lambda_H */
    double f_c, k0, dx;    /* threshold force; Bell k = k0 exp(f dx) */
    double r0;             /* rest length of the harmonic spring law */
    double lj_u, lj_sigma; /* Lennard-Jones depth and minimum distance between
                              non-adjacent beads (lj_u = 0: none) */
    double hi_a;           /* bead radius a of the RPY hydrodynamic interaction
                              (Eqs. 2-3); 0: free draining */
    double vwf_fa, vwf_fb, vwf_xmax;  /* ORA_SPRING_VWF A2 domains: FENE and harmonic
                              spring constants, FENE maximum extension beyond r0 */
} ora_chain;

typedef struct {
    int32_t n_chains;
    int32_t window_steps;      /* S / dt: replica evolution time in steps */
    const ora_chain* chains;
    double dt;
    uint64_t seed;             /* Philox key (low word, high word) */
    int32_t identical_noise;   /* 1: every replica draws the parent's noise */
    int32_t thr_mask;          /* bit q set: threshold criterion on ISF/TSF/RSF */
    int32_t bell_mask;         /* bit q set: Bell criterion on ISF/TSF/RSF */
    double s_min;              /* FENE overextension floor of 1 - H Q^2 / b */
    const int32_t* chain_ids;  /* noise-counter chain id of each chain; NULL = 0, 1, ... */
} ora_problem;

/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11). */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* u = (x + 1/2) 2^-32 in (0, 1). */
double ora_uniform(uint32_t x);
/* u = (m + 1/2) 2^-21 in (0, 1) for a 21-bit field m. */
double ora_uniform21(uint32_t m);
/* Three standard normals for (bead, slot, stream, step, chain): replicas
 * 2j-1 and 2j share the Philox output of counter word 1 = j | stream << 24
 * (the parent: j = 0) and take its two halves. */
void ora_normals3(uint64_t seed, uint32_t bead, uint32_t slot, uint32_t stream,
                  uint32_t step, uint32_t chain, double xi[3]);
/* Unit-mean exponential threshold for a (spring, criterion, chain). */
double ora_exp1(uint64_t seed, uint32_t spring, uint32_t criterion, uint32_t chain);
/* Spring force F(Q) and its signed magnitude along the bond (the tension;
 * |F| for Hooke and FENE, H (|Q| - r0) for the harmonic law with rest length
 * r0); returns 1 when the FENE floor applied. */
int ora_spring_force(int spring, double H, double b, double r0, double s_min, const double Q[3],
                     double F[3], double* tension);
/* Lennard-Jones forces between non-adjacent beads (|i - j| >= 2) of a
 * conformation r [N][3], added to F [N][3]: U = u sum [(s/r)^12 - 2 (s/r)^6]. */
void ora_lj_forces(const ora_chain* ch, const double* r, double* F);
/* Force and signed tension of spring i of a chain under its law (for
 * ORA_SPRING_VWF the law depends on the spring: even springs are A2 domains,
 * odd springs disulfide bonds); returns 1 when a FENE floor applied. */
int ora_chain_spring_force(const ora_chain* ch, int i, double s_min, const double Q[3], double F[3],
                           double* tension);
/* 1 if spring i takes part in the threshold and Bell criteria (every spring,
 * except the disulfide bonds of ORA_SPRING_VWF chains). */
int ora_spring_reacts(const ora_chain* ch, int i);
/* Eqs. 2-3: the RPY diffusion tensor block D_ij / D_0 (D_0 = kT/(6 pi eta a),
 * the single-bead diffusivity) for the separation d = r_j - r_i of two
 * different beads, row-major 3x3. */
void ora_rpy_block(double a, const double d[3], double out[9]);
/* The full 3N x 3N tensor D / D_0 of conformation r [N][3], row-major. */
void ora_rpy_matrix(int N, double a, const double* r, double* D);
/* Lower Cholesky factor L (L L^T = A) of the SPD n x n matrix A, row-major,
 * upper triangle of L zero; returns 1 if A is not positive definite. */
int ora_cholesky(int n, const double* A, double* L);
/* Velocity-gradient tensor kappa (row-major), v = kappa . r. */
void ora_flow_gradient(int flow, double rate, double kappa[9]);
/* One Euler-Maruyama step of Eq. 1 with given noise xi [N][3]; positions r [N][3]. */
int64_t ora_em_step(const ora_chain* ch, double dt, double s_min, double* r, const double* xi);
/* Tension profile [N-1] of a conformation. */
void ora_tensions(const ora_chain* ch, double s_min, const double* r, double* f);

/* Full method over n_steps from global step 0 (see bd_oracle.c for outputs). */
int ora_run(const ora_problem* p, int64_t n_steps, double* pos, double* pos_rep,
            double* rsf, double* tsf, double* lam, int64_t* first_thr, int64_t* first_bell,
            double* exp1, int64_t* overext, int n_threads);

/* The method as ora_run, returning the conformation diagnostics of Eq. 5
 * (Sec. III) at every completed window w (W = n_steps / window_steps), any
 * pointer may be NULL: dbar[W][sum R][3] the bead-mean |COM-frame position
 * difference| between each replica at the window end and the halted parent
 * it was formed from (replicas chain-major); dbead[W][sum N][3] the same per
 * bead, averaged over the chain's replicas; rgz[W][C] the z contribution to
 * the radius of gyration of the halted parent. pos is advanced in place. */
int ora_run_conformation(const ora_problem* p, int64_t n_steps, double* pos, double* dbar,
                         double* dbead, double* rgz, int n_threads);

/* Criteria update for one sampled force value of spring m (used by ora_run;
 * exported so tests can drive kinetics with prescribed force histories). */
void ora_criteria_update(int q, int thr_on, int bell_on, const ora_chain* ch, double f,
                         double dT, int64_t step, double E, double* lam,
                         int64_t* first_thr, int64_t* first_bell);

/* Batch helpers: ctr is [n][4] (word 1 = slot | stream << 24). */
void ora_philox_many(int64_t n, const uint32_t* ctr, const uint32_t key[2], uint32_t* out);
void ora_normals3_many(uint64_t seed, int64_t n, const uint32_t* ctr, double* xi);

/* RSF profiles rsf[W][M] (may be NULL) and their pathwise derivatives with
 * frozen noise drsf[3][W][M] with respect to (rate, b, H) of each chain's own
 * parameters, W = n_steps / window_steps. pos is advanced in place. */
int ora_rsf_tangent(const ora_problem* p, int64_t n_steps, double* pos, double* rsf,
                    double* drsf, int n_threads);

int ora_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
