/*
 * Plain CPU FP64 oracle for replica-averaged Brownian dynamics
 * (Kania, Nguyen, Oztekin & Webb, "Replica-Averaging", arXiv 2206.05851).
 *
 * TEST INFRASTRUCTURE ONLY: the slow, obviously-correct reference for the
 * CUDA path. It is loaded by the tests, the smoke check and the benchmark's
 * CPU-baseline leg, and by nothing in the product library. It shares no
 * source with the CUDA path.
 *
 * What it follows:
 *   - Eq. 1 (Sec. II): Euler-Maruyama update of every bead, taken literally in
 *     the laboratory frame, with the free-draining diffusion tensor of Eq. 2
 *     (D_ij = delta_ij kT/zeta I) or, for chains with a bead radius, the RPY
 *     tensor of Eqs. 2-3 and noise from its lower Cholesky factor.
 *   - Sec. II's collapsed chain: harmonic springs with a rest length and
 *     Lennard-Jones cohesion between non-adjacent beads; the supplement's
 *     coarse-grained vWF chain (A2 domains and disulfide bonds, Table S1).
 *   - Eq. 4 (Sec. II): the instantaneous spring force (ISF) of a spring: the
 *     magnitude of the FENE / Hooke force, the signed force along the bond
 *     for the laws with a rest length.
 *   - Sec. II, "Computing ISF, TSF and RSF": TSF is the mean of per-step
 *     samples over the sampling time S; RSF halts the parent, forms N_R
 *     replicas of it, each with its own noise stream, evolves them for S,
 *     takes ONE force sample per replica at the end and averages over the
 *     replicas, then continues the parent.
 *   - Sec. I and Sec. III (vWF kinetics): events from a force criterion,
 *     either a threshold rupture force or the Bell rate k = k0 exp(f dx / kT)
 *     with the survival integral exp(-int k dt).
 *
 * Readings where the paper is silent (the same readings hold on the GPU side):
 *   FENE law F = H Q / (1 - H Q^2 / b); noise from Philox4x32-10 keyed by
 *   (bead, replica pair | stream << 24, step, chain) with key = seed, six
 *   21-bit uniforms per output and Box-Muller, three normals per slot;
 *   FENE floor s_min on 1 - H Q^2 / b; TSF samples taken after each of the S
 *   updates of a window; hazard of a window force held constant over the
 *   window; first passage when the integrated hazard reaches an Exp(1) draw.
 *
 * Every function here is pinned in the CPU part of the test-suite: by the
 * physics (closed forms, exact Euler laws, stationary densities), by values
 * the paper prints, and Philox by an independent implementation of its
 * definition (the CUDA toolkit's host-side generator). Planted-mistake tests
 * compile copies of this file with one plausible error each and check that
 * its pin fails.
 */
#include "bd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, Salmon et al. SC'11, Sec. 4: a 4-word counter and 2-word   */
/* key; each round multiplies words 0 and 2 by fixed constants, XORs the    */
/* high halves with the other two words and the round key, and permutes;    */
/* the key is bumped by the Weyl constants between rounds.                  */
/* ------------------------------------------------------------------------ */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double ora_uniform(uint32_t x)
{
    return ((double)x + 0.5) * (1.0 / 4294967296.0);
}

/* The random displacement R_i of Eq. 1 needs three standard normals per bead
 * and slot. Replicas 2j-1 and 2j (j >= 1) share one Philox output per (bead,
 * step), counter (bead, j | stream << 24, step, chain); the parent (slot 0)
 * has counter word j = 0. The output's 128 bits give six 21-bit uniforms
 * u = (m + 1/2) 2^-21: m0..m3 the top 21 bits of words 0..3, m4 the low 11
 * bits of word 0 above the low 10 bits of word 1, m5 the same of words 2
 * and 3. Box-Muller (1958) turns the pairs (u0, u1), (u2, u3), (u4, u5) into
 * six independent normals z_k = r (cos, sin)(2 pi u_angle),
 * r = sqrt(-2 ln u_radius); the odd slot (and the parent) takes z0, z1, z2,
 * the even replica slot z3, z4, z5. */
double ora_uniform21(uint32_t m)
{
    return ((double)m + 0.5) * (1.0 / 2097152.0);
}

void ora_normals3(uint64_t seed, uint32_t bead, uint32_t slot, uint32_t stream,
                  uint32_t step, uint32_t chain, double xi[3])
{
    const uint32_t pair = (slot + 1u) / 2u;
    const int second = slot != 0u && slot % 2u == 0u;
    uint32_t ctr[4] = { bead, pair | (stream << 24), step, chain };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t x[4];
    ora_philox4x32_10(ctr, key, x);
    const uint32_t m[6] = { x[0] >> 11, x[1] >> 11, x[2] >> 11, x[3] >> 11,
                            ((x[0] & 0x7FFu) << 10) | (x[1] & 0x3FFu),
                            ((x[2] & 0x7FFu) << 10) | (x[3] & 0x3FFu) };
    double z[6];
    for (int k = 0; k < 3; ++k) {
        const double rho = sqrt(-2.0 * log(ora_uniform21(m[2 * k])));
        const double theta = 2.0 * ORA_PI * ora_uniform21(m[2 * k + 1]);
        z[2 * k] = rho * cos(theta);
        z[2 * k + 1] = rho * sin(theta);
    }
    for (int d = 0; d < 3; ++d) xi[d] = z[3 * second + d];
}

/* Exp(1) threshold of the first-passage test: E = -ln u, one uniform from the
 * second Philox stream, counter (spring, stream << 24, criterion, chain). */
double ora_exp1(uint64_t seed, uint32_t spring, uint32_t criterion, uint32_t chain)
{
    uint32_t ctr[4] = { spring, (uint32_t)ORA_STREAM_EXP1 << 24, criterion, chain };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t x[4];
    ora_philox4x32_10(ctr, key, x);
    return -log(ora_uniform(x[0]));
}

/* ------------------------------------------------------------------------ */
/* Spring laws. Hookean: F = H Q. FENE (Warner): F = H Q / (1 - H Q^2 / b),   */
/* the gradient of U = -(b/2) ln(1 - H Q^2 / b). F is the force on the lower */
/* bead of the spring, pointing towards the upper bead.                      */
/* ------------------------------------------------------------------------ */
int ora_spring_force(int spring, double H, double b, double r0, double s_min, const double Q[3],
                     double F[3], double* tension)
{
    double q2 = Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2];
    double coef = H;
    int floored = 0;
    if (spring == ORA_SPRING_FENE) {
        double s = 1.0 - H * q2 / b;
        if (s < s_min) { s = s_min; floored = 1; }
        coef = H / s;
    }
    if (spring == ORA_SPRING_HARMONIC) {
        /* Sec. II: U_s = (kappa/2) (|Q| - 2a)^2, force kappa (|Q| - r0) along Q */
        const double q = sqrt(q2);
        coef = q > 0.0 ? H * (q - r0) / q : 0.0;
        F[0] = coef * Q[0];
        F[1] = coef * Q[1];
        F[2] = coef * Q[2];
        if (tension) *tension = H * (q - r0);          /* Eq. 4, signed */
        return 0;
    }
    F[0] = coef * Q[0];
    F[1] = coef * Q[1];
    F[2] = coef * Q[2];
    if (tension) *tension = coef * sqrt(q2);
    return floored;
}

/* The coarse-grained vWF chain (supplementary material, Table S1): a monomer
 * is two beads joined by an A2 domain, a FENE spring in parallel with a
 * stiffer harmonic spring; monomers are joined by disulfide bonds, stiff
 * harmonic springs. Spring i joins beads i and i+1, so even springs are A2
 * domains and odd springs disulfide bonds. With x = |Q| - r0 the extension
 * beyond the rest length:
 *   A2:        f = f_B x + f_A x / (1 - x^2 / x_max^2)   (the sum of the two
 *              springs' forces, the force on the domain),
 *   disulfide: f = H x,
 * both along Q and signed as Eq. 4; the FENE denominator is floored at s_min
 * like the FENE law above. */
int ora_chain_spring_force(const ora_chain* ch, int i, double s_min, const double Q[3], double F[3],
                           double* tension)
{
    if (ch->spring != ORA_SPRING_VWF)
        return ora_spring_force(ch->spring, ch->H, ch->b, ch->r0, s_min, Q, F, tension);
    const double q = sqrt(Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2]);
    const double x = q - ch->r0;
    double f;
    int floored = 0;
    if (i % 2 == 0) {
        double s = 1.0 - x * x / (ch->vwf_xmax * ch->vwf_xmax);
        if (s < s_min) { s = s_min; floored = 1; }
        f = ch->vwf_fb * x + ch->vwf_fa * x / s;
    } else {
        f = ch->H * x;
    }
    const double coef = q > 0.0 ? f / q : 0.0;
    F[0] = coef * Q[0];
    F[1] = coef * Q[1];
    F[2] = coef * Q[2];
    if (tension) *tension = f;
    return floored;
}

int ora_spring_reacts(const ora_chain* ch, int i)
{
    return ch->spring != ORA_SPRING_VWF || i % 2 == 0;
}

/* Sec. II: U_LJ = u sum_{ij} [(2a/r_ij)^12 - 2 (2a/r_ij)^6] over non-adjacent
 * beads; the force on bead i from bead j is -dU/dr_i = (dU/dr) r_ij / r with
 * r_ij = r_j - r_i and dU/dr = (12 u / r) [(s/r)^6 - (s/r)^12]. */
void ora_lj_forces(const ora_chain* ch, const double* r, double* F)
{
    if (!(ch->lj_u > 0.0)) return;
    const int N = ch->n_beads;
    const double s2 = ch->lj_sigma * ch->lj_sigma;
    for (int i = 0; i < N; ++i)
        for (int j = i + 2; j < N; ++j) {
            const double d[3] = { r[3 * j] - r[3 * i], r[3 * j + 1] - r[3 * i + 1],
                                  r[3 * j + 2] - r[3 * i + 2] };
            const double rr = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            const double x6 = (s2 / rr) * (s2 / rr) * (s2 / rr);
            const double dUdr_over_r = 12.0 * ch->lj_u * (x6 - x6 * x6) / rr;
            for (int k = 0; k < 3; ++k) {
                F[3 * i + k] += dUdr_over_r * d[k];
                F[3 * j + k] -= dUdr_over_r * d[k];
            }
        }
}

/* Eq. 3 divided by D_0 = kT/(6 pi eta a): for r = |d| >= 2a
 *   (3a / 4r) [(1 + 2a^2/(3r^2)) I + (1 - 2a^2/r^2) d d / r^2],
 * and for r < 2a (overlapping beads)
 *   (3a / 4r) (r / 2a) [(8/3 - 3r/(4a)) I + (r / 4a) d d / r^2]. */
void ora_rpy_block(double a, const double d[3], double out[9])
{
    const double rr = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double r = sqrt(rr);
    const double pre = 3.0 * a / (4.0 * r);
    double ci, cd;                       /* coefficients of I and of d d / r^2 */
    if (r >= 2.0 * a) {
        ci = pre * (1.0 + 2.0 * a * a / (3.0 * rr));
        cd = pre * (1.0 - 2.0 * a * a / rr);
    } else {
        ci = pre * (r / (2.0 * a)) * (8.0 / 3.0 - 3.0 * r / (4.0 * a));
        cd = pre * (r / (2.0 * a)) * (r / (4.0 * a));
    }
    for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y)
            out[3 * x + y] = (x == y ? ci : 0.0) + cd * d[x] * d[y] / rr;
}

/* Eq. 2 on the diagonal blocks (D_ii = D_0 I), Eq. 3 off it. */
void ora_rpy_matrix(int N, double a, const double* r, double* D)
{
    const int n = 3 * N;
    for (int i = 0; i < n * n; ++i) D[i] = 0.0;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            double blk[9];
            if (i == j) {
                for (int k = 0; k < 9; ++k) blk[k] = (k % 4 == 0) ? 1.0 : 0.0;
            } else {
                const double d[3] = { r[3 * j] - r[3 * i], r[3 * j + 1] - r[3 * i + 1],
                                      r[3 * j + 2] - r[3 * i + 2] };
                ora_rpy_block(a, d, blk);
            }
            for (int x = 0; x < 3; ++x)
                for (int y = 0; y < 3; ++y)
                    D[(3 * i + x) * n + 3 * j + y] = blk[3 * x + y];
        }
}

/* Cholesky-Banachiewicz, row by row: L_ij = (A_ij - sum_{k<j} L_ik L_jk) / L_jj
 * for j < i, L_ii = sqrt(A_ii - sum_{k<i} L_ik^2). */
int ora_cholesky(int n, const double* A, double* L)
{
    for (int i = 0; i < n * n; ++i) L[i] = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            if (i == j) {
                if (!(s > 0.0)) return 1;
                L[i * n + i] = sqrt(s);
            } else {
                L[i * n + j] = s / L[j * n + j];
            }
        }
    return 0;
}

/* Homogeneous flows v = kappa . r. Shear as in Sec. II: v = gdot z x_hat
 * (x flow direction, z gradient direction). Uniaxial elongation:
 * rate * diag(1, -1/2, -1/2). Planar elongation: rate * diag(1, -1, 0). */
void ora_flow_gradient(int flow, double rate, double kappa[9])
{
    for (int i = 0; i < 9; ++i) kappa[i] = 0.0;
    switch (flow) {
    case ORA_FLOW_SHEAR:    kappa[0 * 3 + 2] = rate; break;
    case ORA_FLOW_UNIAXIAL: kappa[0] = rate; kappa[4] = -0.5 * rate; kappa[8] = -0.5 * rate; break;
    case ORA_FLOW_PLANAR:   kappa[0] = rate; kappa[4] = -rate; break;
    default: break;
    }
}

/* Eq. 1 with Eq. 2 (free draining): each bead moves with the solvent velocity
 * at its position plus D/kT times the spring force on it, plus a random
 * displacement of covariance 2 D dt. kT = 1 and D = kT/zeta = 1/4 in Hookean
 * units. The spring force on bead i is F_i - F_{i-1} (F_i: force of spring i,
 * which joins beads i and i+1; F_{-1} = F_{N-1} = 0). Every drift is taken at
 * time t, so the increments are formed first and applied afterwards.
 * With hydrodynamic interaction (hi_a > 0, Eqs. 1-3) the drift is
 * (1/kT) sum_j D_ij F_j and the random displacement sqrt(2 dt) B xi with
 * B B^T = D: here D = D_0 W (W the tensor of ora_rpy_matrix, D_0 = 1/4) and B
 * = sqrt(D_0) L, L the lower Cholesky factor of W. RPY is divergence-free,
 * so Eq. 1 needs no drift correction.
 * Returns the number of springs whose FENE floor applied. */
int64_t ora_em_step(const ora_chain* ch, double dt, double s_min, double* r, const double* xi)
{
    const double D = 0.25, kT = 1.0;
    const int N = ch->n_beads;
    double kappa[9];
    ora_flow_gradient(ch->flow, ch->rate, kappa);
    double* F = (double*)calloc(3 * (size_t)N, sizeof(double));
    double* inc = (double*)calloc(3 * (size_t)N, sizeof(double));
    int64_t floored = 0;
    for (int i = 0; i + 1 < N; ++i) {
        double Q[3] = { r[3 * (i + 1) + 0] - r[3 * i + 0],
                        r[3 * (i + 1) + 1] - r[3 * i + 1],
                        r[3 * (i + 1) + 2] - r[3 * i + 2] };
        floored += ora_chain_spring_force(ch, i, s_min, Q, &F[3 * i], NULL);
    }
    double* Flj = (double*)calloc(3 * (size_t)N, sizeof(double));
    ora_lj_forces(ch, r, Flj);
    const double amp = sqrt(2.0 * D * dt);
    /* total force on each bead */
    double* Fb = (double*)calloc(3 * (size_t)N, sizeof(double));
    for (int i = 0; i < N; ++i)
        for (int d = 0; d < 3; ++d) {
            double fb = Flj[3 * i + d];
            if (i + 1 < N) fb += F[3 * i + d];
            if (i > 0)     fb -= F[3 * (i - 1) + d];
            Fb[3 * i + d] = fb;
        }
    /* mobility-weighted force and correlated noise (free draining: W = I) */
    const int n = 3 * N;
    double* drift = (double*)calloc((size_t)n, sizeof(double));
    double* noise = (double*)calloc((size_t)n, sizeof(double));
    if (ch->hi_a > 0.0) {
        double* W = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
        double* Lc = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
        ora_rpy_matrix(N, ch->hi_a, r, W);
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) drift[p] += W[p * n + q] * Fb[q];
        if (ora_cholesky(n, W, Lc)) {
            for (int p = 0; p < n; ++p) noise[p] = NAN;   /* not positive definite */
        } else {
            for (int p = 0; p < n; ++p)
                for (int q = 0; q <= p; ++q) noise[p] += Lc[p * n + q] * xi[q];
        }
        free(W);
        free(Lc);
    } else {
        for (int p = 0; p < n; ++p) { drift[p] = Fb[p]; noise[p] = xi[p]; }
    }
    for (int i = 0; i < N; ++i) {
        for (int d = 0; d < 3; ++d) {
            double v = kappa[3 * d + 0] * r[3 * i + 0] + kappa[3 * d + 1] * r[3 * i + 1]
                     + kappa[3 * d + 2] * r[3 * i + 2];
            inc[3 * i + d] = (v + (D / kT) * drift[3 * i + d]) * dt + amp * noise[3 * i + d];
        }
    }
    for (int i = 0; i < 3 * N; ++i) r[i] += inc[i];
    free(inc);
    free(F);
    free(Flj);
    free(Fb);
    free(drift);
    free(noise);
    return floored;
}

/* Eq. 4: the instantaneous force of each spring, as a magnitude. */
void ora_tensions(const ora_chain* ch, double s_min, const double* r, double* f)
{
    for (int i = 0; i + 1 < ch->n_beads; ++i) {
        double Q[3] = { r[3 * (i + 1) + 0] - r[3 * i + 0],
                        r[3 * (i + 1) + 1] - r[3 * i + 1],
                        r[3 * (i + 1) + 2] - r[3 * i + 2] };
        double F[3];
        ora_chain_spring_force(ch, i, s_min, Q, F, &f[i]);
    }
}

/* One sampled force f of one spring under criterion q, attributed to an
 * interval dT ending at global step `step`:
 *   threshold: first step with f >= f_c (ties count);
 *   Bell: hazard += k0 exp(f dx) dT (force held constant over dT); first
 *   passage at the first step where the integrated hazard reaches E. */
void ora_criteria_update(int q, int thr_on, int bell_on, const ora_chain* ch, double f,
                         double dT, int64_t step, double E, double* lam,
                         int64_t* first_thr, int64_t* first_bell)
{
    (void)q;
    if (thr_on && *first_thr < 0 && f >= ch->f_c) *first_thr = step;
    if (bell_on) {
        *lam += ch->k0 * exp(f * ch->dx) * dT;
        if (*first_bell < 0 && *lam >= E) *first_bell = step;
    }
}

/* Batch forms of the two generators above, for tests that need many draws. */
void ora_philox_many(int64_t n, const uint32_t* ctr, const uint32_t key[2], uint32_t* out)
{
    for (int64_t j = 0; j < n; ++j) ora_philox4x32_10(&ctr[4 * j], key, &out[4 * j]);
}

void ora_normals3_many(uint64_t seed, int64_t n, const uint32_t* ctr, double* xi)
{
    for (int64_t j = 0; j < n; ++j)
        ora_normals3(seed, ctr[4 * j + 0], ctr[4 * j + 1] & 0xFFFFFFu, ctr[4 * j + 1] >> 24,
                     ctr[4 * j + 2], ctr[4 * j + 3], &xi[3 * j]);
}

/* ------------------------------------------------------------------------ */
/* Pathwise derivatives with frozen noise (forward-mode tangents).          */
/* Parameters theta = (rate, b, H) of every chain. Each slot carries, beside */
/* its positions r, the three tangents dr/dtheta_j; the Euler map of Eq. 1   */
/* is differentiated with the noise held fixed, and a spawned replica copies */
/* the parent's tangents with its positions. The RSF tangent follows from    */
/* the tension f = |F(Q)| of each replica at the window end.                 */
/* ------------------------------------------------------------------------ */

/* Spring-law derivatives at connector Q: force F = c Q with c = H / s,
 * s = 1 - H Q^2 / b (Hooke: c = H). dF = c dQ + (dc/dq2) 2 (Q.dQ) Q for a
 * change of Q; dc/dH and dc/db for a change of the parameters (zero for b,
 * and constant in Q, once the floor applies). */
static void ora_spring_partials(const ora_chain* ch, double s_min, const double Q[3],
                                double* c, double* dc_dq2, double* dc_dH, double* dc_db)
{
    const double q2 = Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2];
    if (ch->spring != ORA_SPRING_FENE) {
        *c = ch->H; *dc_dq2 = 0.0; *dc_dH = 1.0; *dc_db = 0.0;
        return;
    }
    double s = 1.0 - ch->H * q2 / ch->b;
    if (s < s_min) {
        *c = ch->H / s_min; *dc_dq2 = 0.0; *dc_dH = 1.0 / s_min; *dc_db = 0.0;
        return;
    }
    *c = ch->H / s;
    *dc_dq2 = ch->H * ch->H / (ch->b * s * s);               /* -H/s^2 * ds/dq2 */
    *dc_dH = 1.0 / s + ch->H * q2 / (ch->b * s * s);         /* 1/s^2 */
    *dc_db = -ch->H * ch->H * q2 / (ch->b * ch->b * s * s);  /* -H/s^2 * ds/db  */
}

/* Directional derivative of the spring force: dF for a connector change dQ
 * and parameter changes (dH, db). */
static void ora_force_tangent(const ora_chain* ch, double s_min, const double Q[3],
                              const double dQ[3], double dH, double db, double dF[3])
{
    double c, dcq, dcH, dcb;
    ora_spring_partials(ch, s_min, Q, &c, &dcq, &dcH, &dcb);
    const double qdq = Q[0] * dQ[0] + Q[1] * dQ[1] + Q[2] * dQ[2];
    const double dc = dcq * 2.0 * qdq + dcH * dH + dcb * db;
    for (int d = 0; d < 3; ++d) dF[d] = c * dQ[d] + dc * Q[d];
}

/* One Eq. 1 step of positions r and of their tangents tr[3][N][3] (for rate,
 * b, H), noise xi frozen. The tangent of a drift term is taken at time t. */
static int64_t ora_em_step_tangent(const ora_chain* ch, double dt, double s_min, double* r,
                                   double* tr, const double* xi)
{
    const double D = 0.25, kT = 1.0;
    const int N = ch->n_beads;
    double kappa[9], khat[9];
    ora_flow_gradient(ch->flow, ch->rate, kappa);
    ora_flow_gradient(ch->flow, 1.0, khat);                 /* d kappa / d rate */
    double* dr = (double*)calloc(3 * (size_t)N * 3, sizeof(double));
    for (int j = 0; j < 3; ++j) {
        const double dH = j == 2 ? 1.0 : 0.0, db = j == 1 ? 1.0 : 0.0;
        double* t = tr + 3 * (size_t)N * j;
        double* F = (double*)calloc(3 * (size_t)N, sizeof(double));
        for (int i = 0; i + 1 < N; ++i) {
            double Q[3], dQ[3];
            for (int d = 0; d < 3; ++d) {
                Q[d] = r[3 * (i + 1) + d] - r[3 * i + d];
                dQ[d] = t[3 * (i + 1) + d] - t[3 * i + d];
            }
            ora_force_tangent(ch, s_min, Q, dQ, dH, db, &F[3 * i]);
        }
        for (int i = 0; i < N; ++i) {
            for (int d = 0; d < 3; ++d) {
                double dfs = 0.0;
                if (i + 1 < N) dfs += F[3 * i + d];
                if (i > 0)     dfs -= F[3 * (i - 1) + d];
                double dv = kappa[3 * d + 0] * t[3 * i + 0] + kappa[3 * d + 1] * t[3 * i + 1]
                          + kappa[3 * d + 2] * t[3 * i + 2];
                if (j == 0)
                    dv += khat[3 * d + 0] * r[3 * i + 0] + khat[3 * d + 1] * r[3 * i + 1]
                        + khat[3 * d + 2] * r[3 * i + 2];
                dr[(3 * (size_t)N) * j + 3 * i + d] = (dv + (D / kT) * dfs) * dt;
            }
        }
        free(F);
    }
    const int64_t fl = ora_em_step(ch, dt, s_min, r, xi);
    for (size_t k = 0; k < 3 * (size_t)N * 3; ++k) tr[k] += dr[k];
    free(dr);
    return fl;
}

/* Tension f = c |Q| of spring i and its tangent for (dQ, dH, db). */
static double ora_tension_tangent(const ora_chain* ch, double s_min, const double Q[3],
                                  const double dQ[3], double dH, double db)
{
    double c, dcq, dcH, dcb;
    ora_spring_partials(ch, s_min, Q, &c, &dcq, &dcH, &dcb);
    const double q = sqrt(Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2]);
    if (q == 0.0) return 0.0;
    const double qdq = Q[0] * dQ[0] + Q[1] * dQ[1] + Q[2] * dQ[2];
    const double dc = dcq * 2.0 * qdq + dcH * dH + dcb * db;
    return dc * q + c * qdq / q;
}

/* RSF profiles and their tangents d RSF[w][m] / d theta_j, written to
 * drsf[j][w][M] (j = 0 rate, 1 b, 2 H), for the same run as ora_run
 * (criteria are not evaluated). pos is advanced in place. */
int ora_rsf_tangent(const ora_problem* p, int64_t n_steps, double* pos, double* rsf,
                    double* drsf, int n_threads)
{
    const int C = p->n_chains;
    const int S = p->window_steps;
    if (C <= 0 || S <= 0 || n_steps < 0) return 1;
    for (int c = 0; c < C; ++c)      /* tangents of the Hooke and FENE laws only */
        if (p->chains[c].spring == ORA_SPRING_HARMONIC || p->chains[c].spring == ORA_SPRING_VWF ||
            p->chains[c].lj_u > 0.0 ||
            p->chains[c].hi_a > 0.0) return 1;
    int64_t* bead_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(C + 1));
    int64_t* spr_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(C + 1));
    bead_off[0] = spr_off[0] = 0;
    for (int c = 0; c < C; ++c) {
        bead_off[c + 1] = bead_off[c] + p->chains[c].n_beads;
        spr_off[c + 1] = spr_off[c] + p->chains[c].n_beads - 1;
    }
    const int64_t M = spr_off[C];
    const int64_t W = n_steps / S;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#else
    (void)n_threads;
#endif
    for (int c = 0; c < C; ++c) {
        const ora_chain* ch = &p->chains[c];
        const int N = ch->n_beads, R = ch->n_replicas;
        const uint32_t cid = p->chain_ids ? (uint32_t)p->chain_ids[c] : (uint32_t)c;
        const size_t sz = 3 * (size_t)N;
        double* par = pos + 3 * bead_off[c];
        double* tpar = (double*)calloc(3 * sz, sizeof(double));
        double* rk = (double*)malloc(sizeof(double) * sz);
        double* tk = (double*)malloc(sizeof(double) * 3 * sz);
        double* xi = (double*)malloc(sizeof(double) * sz);
        double* acc = (double*)malloc(sizeof(double) * 4 * (size_t)N);
        for (int64_t t = 0; t < n_steps; ) {
            const int64_t w = t / S;
            const int Sw = (int)((n_steps - t) < S ? (n_steps - t) : S);
            for (int i = 0; i < 4 * N; ++i) acc[i] = 0.0;
            for (int k = 1; k <= R; ++k) {
                memcpy(rk, par, sizeof(double) * sz);
                memcpy(tk, tpar, sizeof(double) * 3 * sz);
                const uint32_t slot = p->identical_noise ? 0u : (uint32_t)k;
                for (int s = 0; s < Sw; ++s) {
                    for (int i = 0; i < N; ++i)
                        ora_normals3(p->seed, (uint32_t)i, slot, ORA_STREAM_BD,
                                     (uint32_t)(t + s), cid, &xi[3 * i]);
                    ora_em_step_tangent(ch, p->dt, p->s_min, rk, tk, xi);
                }
                if (Sw == S) {
                    for (int i = 0; i + 1 < N; ++i) {
                        double Q[3];
                        for (int d = 0; d < 3; ++d) Q[d] = rk[3 * (i + 1) + d] - rk[3 * i + d];
                        double F[3], f;
                        ora_spring_force(ch->spring, ch->H, ch->b, ch->r0, p->s_min, Q, F, &f);
                        acc[i] += f;
                        for (int j = 0; j < 3; ++j) {
                            double dQ[3];
                            const double* tj = tk + sz * j;
                            for (int d = 0; d < 3; ++d) dQ[d] = tj[3 * (i + 1) + d] - tj[3 * i + d];
                            acc[(size_t)N * (j + 1) + i] += ora_tension_tangent(
                                ch, p->s_min, Q, dQ, j == 2 ? 1.0 : 0.0, j == 1 ? 1.0 : 0.0);
                        }
                    }
                }
            }
            for (int s = 0; s < Sw; ++s) {
                for (int i = 0; i < N; ++i)
                    ora_normals3(p->seed, (uint32_t)i, 0u, ORA_STREAM_BD, (uint32_t)(t + s), cid,
                                 &xi[3 * i]);
                ora_em_step_tangent(ch, p->dt, p->s_min, par, tpar, xi);
            }
            if (Sw == S) {
                for (int i = 0; i + 1 < N; ++i) {
                    const int64_t m = spr_off[c] + i;
                    if (rsf) rsf[w * M + m] = acc[i] / R;
                    for (int j = 0; j < 3; ++j)
                        drsf[((int64_t)j * W + w) * M + m] = acc[(size_t)N * (j + 1) + i] / R;
                }
            }
            t += Sw;
        }
        free(tpar); free(rk); free(tk); free(xi); free(acc);
    }
    free(bead_off); free(spr_off);
    return 0;
}

int ora_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* The method, chain by chain, in the order of Sec. II:                     */
/*   at every sampling time t_w = w S (w = 0, 1, ...):                      */
/*     halt the parent; copy it into N_R replicas; evolve replica k for S   */
/*     steps with its own noise stream (slot k); sample the force of every  */
/*     spring once at the end; RSF = mean over replicas;                    */
/*     continue the parent for S steps (slot 0), sampling its force every   */
/*     step (ISF) and averaging the samples over the window (TSF).          */
/* Global step t keys the noise of the update t -> t+1 for every slot, so a */
/* replica and the parent advance through the same step counter.           */
/*                                                                          */
/* Arrays (M = sum over chains of N_c - 1, springs of chain c at spr_off[c]):*/
/*   pos        in/out [sum N][3] parent positions, laboratory frame        */
/*   pos_rep    out [sum R N][3] replica positions at the end, or NULL      */
/*   rsf, tsf   out [n_steps / S][M] window profiles, or NULL               */
/*   lam        in/out [3][M] integrated Bell hazard per criterion          */
/*   first_thr, first_bell in/out [3][M] first event step, -1 if none       */
/*   exp1       out [3][M] Exp(1) thresholds, or NULL                       */
/*   overext    out [n_chains] FENE-floor applications (all slots)          */
/* A run that ends inside a window evolves the replicas and the parent      */
/* through the partial window and takes no window sample.                   */
/* ------------------------------------------------------------------------ */
/* Conformation difference of Eq. 5 (Sec. III) between a replica rk and the
 * halted parent P_c it was formed from, both in their own centre-of-mass
 * frames: D(j, i) = |rhat_j^i(S, k) - rhat_j^i(P_c)|; dsum[j] = sum over beads.
 * acc (may be NULL) receives += D(j, i). */
static void eq5_difference(int N, const double* rk, const double* parent, double dsum[3],
                           double* acc)
{
    double ck[3] = {0, 0, 0}, cp[3] = {0, 0, 0};
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < 3; ++j) { ck[j] += rk[3 * i + j]; cp[j] += parent[3 * i + j]; }
    for (int j = 0; j < 3; ++j) { ck[j] /= N; cp[j] /= N; dsum[j] = 0.0; }
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < 3; ++j) {
            const double d = fabs((rk[3 * i + j] - ck[j]) - (parent[3 * i + j] - cp[j]));
            dsum[j] += d;
            if (acc) acc[3 * i + j] += d;
        }
}

/* z contribution to the radius of gyration of a conformation (Sec. III):
 * sqrt(mean over beads of (z_i - z_cm)^2). */
static double radius_gyration_z(int N, const double* r)
{
    double cz = 0.0;
    for (int i = 0; i < N; ++i) cz += r[3 * i + 2];
    cz /= N;
    double s2 = 0.0;
    for (int i = 0; i < N; ++i) s2 += (r[3 * i + 2] - cz) * (r[3 * i + 2] - cz);
    return sqrt(s2 / N);
}

static int run_impl(const ora_problem* p, int64_t n_steps, double* pos, double* pos_rep,
                    double* rsf, double* tsf, double* lam, int64_t* first_thr,
                    int64_t* first_bell, double* exp1, int64_t* overext, double* dbar,
                    double* dbead, double* rgz, int n_threads)
{
    const int C = p->n_chains;
    const int S = p->window_steps;
    if (C <= 0 || S <= 0 || n_steps < 0) return 1;
    int64_t* bead_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(C + 1));
    int64_t* spr_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(C + 1));
    int64_t* rep_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(C + 1));
    int64_t* repc_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(C + 1));
    bead_off[0] = spr_off[0] = rep_off[0] = repc_off[0] = 0;
    for (int c = 0; c < C; ++c) {
        bead_off[c + 1] = bead_off[c] + p->chains[c].n_beads;
        spr_off[c + 1] = spr_off[c] + p->chains[c].n_beads - 1;
        rep_off[c + 1] = rep_off[c] + (int64_t)p->chains[c].n_replicas * p->chains[c].n_beads;
        repc_off[c + 1] = repc_off[c] + p->chains[c].n_replicas;
    }
    const int64_t M = spr_off[C];
    const int64_t NB = bead_off[C], NR = repc_off[C];

#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#else
    (void)n_threads;
#endif
    for (int c = 0; c < C; ++c) {
        const ora_chain* ch = &p->chains[c];
        const int N = ch->n_beads, R = ch->n_replicas;
        const uint32_t cid = p->chain_ids ? (uint32_t)p->chain_ids[c] : (uint32_t)c;
        const int64_t so = spr_off[c];
        double* parent = pos + 3 * bead_off[c];
        double* rep = (double*)malloc(sizeof(double) * 3 * (size_t)N * (size_t)R);
        double* xi = (double*)malloc(sizeof(double) * 3 * (size_t)N);
        double* f = (double*)malloc(sizeof(double) * (size_t)N);
        double* rsum = (double*)malloc(sizeof(double) * (size_t)N);
        double* tsum = (double*)malloc(sizeof(double) * (size_t)N);
        double* E = (double*)malloc(sizeof(double) * 3 * (size_t)N);
        double* dacc = (double*)malloc(sizeof(double) * 3 * (size_t)N);
        int64_t nover = 0;

        for (int q = 0; q < 3; ++q)
            for (int i = 0; i + 1 < N; ++i) {
                E[q * N + i] = ora_exp1(p->seed, (uint32_t)i, (uint32_t)q, cid);
                if (exp1) exp1[q * M + so + i] = E[q * N + i];
            }

        for (int k = 0; k < R; ++k)
            memcpy(rep + 3 * (size_t)N * k, parent, sizeof(double) * 3 * (size_t)N);

        for (int64_t t = 0; t < n_steps; ) {
            const int64_t w = t / S;
            const int Sw = (int)((n_steps - t) < S ? (n_steps - t) : S);

            /* RSF: halt the parent, spawn replicas, evolve them for S. */
            for (int i = 0; i + 1 < N; ++i) rsum[i] = 0.0;
            for (int i = 0; i < 3 * N; ++i) dacc[i] = 0.0;
            for (int k = 1; k <= R; ++k) {
                double* rk = rep + 3 * (size_t)N * (k - 1);
                memcpy(rk, parent, sizeof(double) * 3 * (size_t)N);
                const uint32_t slot = p->identical_noise ? 0u : (uint32_t)k;
                for (int s = 0; s < Sw; ++s) {
                    for (int i = 0; i < N; ++i)
                        ora_normals3(p->seed, (uint32_t)i, slot, ORA_STREAM_BD,
                                     (uint32_t)(t + s), cid, &xi[3 * i]);
                    nover += ora_em_step(ch, p->dt, p->s_min, rk, xi);
                }
                if (Sw == S) {
                    ora_tensions(ch, p->s_min, rk, f);
                    for (int i = 0; i + 1 < N; ++i) rsum[i] += f[i];
                    if (dbar || dbead) {   /* Eq. 5 against the still-halted parent */
                        double dsum[3];
                        eq5_difference(N, rk, parent, dsum, dbead ? dacc : NULL);
                        if (dbar)
                            for (int j = 0; j < 3; ++j)
                                dbar[(w * NR + repc_off[c] + k - 1) * 3 + j] = dsum[j] / N;
                    }
                }
            }
            if (Sw == S) {
                if (dbead)
                    for (int i = 0; i < N; ++i)
                        for (int j = 0; j < 3; ++j)
                            dbead[(w * NB + bead_off[c] + i) * 3 + j] = dacc[3 * i + j] / R;
                if (rgz) rgz[w * C + c] = radius_gyration_z(N, parent);
            }

            /* Continue the parent through the same S steps. */
            for (int i = 0; i + 1 < N; ++i) tsum[i] = 0.0;
            for (int s = 0; s < Sw; ++s) {
                for (int i = 0; i < N; ++i)
                    ora_normals3(p->seed, (uint32_t)i, 0u, ORA_STREAM_BD, (uint32_t)(t + s),
                                 cid, &xi[3 * i]);
                nover += ora_em_step(ch, p->dt, p->s_min, parent, xi);
                ora_tensions(ch, p->s_min, parent, f);
                for (int i = 0; i + 1 < N; ++i) {
                    tsum[i] += f[i];
                    const int64_t m = so + i;
                    if (ora_spring_reacts(ch, i))
                        ora_criteria_update(ORA_ISF, (p->thr_mask >> ORA_ISF) & 1,
                                            (p->bell_mask >> ORA_ISF) & 1, ch, f[i], p->dt,
                                            t + s + 1, E[ORA_ISF * N + i],
                                            &lam[ORA_ISF * M + m], &first_thr[ORA_ISF * M + m],
                                            &first_bell[ORA_ISF * M + m]);
                }
            }

            if (Sw == S) {
                const double dT = S * p->dt;
                for (int i = 0; i + 1 < N; ++i) {
                    const int64_t m = so + i;
                    const double fr = rsum[i] / R;
                    const double ft = tsum[i] / S;
                    if (rsf) rsf[w * M + m] = fr;
                    if (tsf) tsf[w * M + m] = ft;
                    if (!ora_spring_reacts(ch, i)) continue;
                    ora_criteria_update(ORA_TSF, (p->thr_mask >> ORA_TSF) & 1,
                                        (p->bell_mask >> ORA_TSF) & 1, ch, ft, dT, t + S,
                                        E[ORA_TSF * N + i],
                                        &lam[ORA_TSF * M + m], &first_thr[ORA_TSF * M + m],
                                        &first_bell[ORA_TSF * M + m]);
                    ora_criteria_update(ORA_RSF, (p->thr_mask >> ORA_RSF) & 1,
                                        (p->bell_mask >> ORA_RSF) & 1, ch, fr, dT, t + S,
                                        E[ORA_RSF * N + i],
                                        &lam[ORA_RSF * M + m], &first_thr[ORA_RSF * M + m],
                                        &first_bell[ORA_RSF * M + m]);
                }
            }
            t += Sw;
        }

        if (pos_rep)
            memcpy(pos_rep + 3 * rep_off[c], rep, sizeof(double) * 3 * (size_t)N * (size_t)R);
        overext[c] = nover;
        free(rep); free(xi); free(f); free(rsum); free(tsum); free(E); free(dacc);
    }
    free(bead_off); free(spr_off); free(rep_off); free(repc_off);
    return 0;
}

int ora_run(const ora_problem* p, int64_t n_steps, double* pos, double* pos_rep,
            double* rsf, double* tsf, double* lam, int64_t* first_thr, int64_t* first_bell,
            double* exp1, int64_t* overext, int n_threads)
{
    return run_impl(p, n_steps, pos, pos_rep, rsf, tsf, lam, first_thr, first_bell, exp1,
                    overext, NULL, NULL, NULL, n_threads);
}

int ora_run_conformation(const ora_problem* p, int64_t n_steps, double* pos, double* dbar,
                         double* dbead, double* rgz, int n_threads)
{
    if (p->n_chains <= 0) return 1;
    int64_t M = 0;
    for (int c = 0; c < p->n_chains; ++c) M += p->chains[c].n_beads - 1;
    double* lam = (double*)calloc((size_t)(3 * M + 1), sizeof(double));
    int64_t* ft = (int64_t*)malloc(sizeof(int64_t) * (size_t)(3 * M + 1));
    int64_t* fb = (int64_t*)malloc(sizeof(int64_t) * (size_t)(3 * M + 1));
    int64_t* ov = (int64_t*)malloc(sizeof(int64_t) * (size_t)p->n_chains);
    for (int64_t m = 0; m < 3 * M; ++m) ft[m] = fb[m] = -1;
    const int rc = run_impl(p, n_steps, pos, NULL, NULL, NULL, lam, ft, fb, NULL, ov, dbar,
                            dbead, rgz, n_threads);
    free(lam); free(ft); free(fb); free(ov);
    return rc;
}
