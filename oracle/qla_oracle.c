/*
 * Plain FP64 CPU oracle for the qubit lattice algorithm (QLA) of
 * "Qubit Lattice Algorithm Simulations of Maxwell's Equations for Scattering
 * from Anisotropic Dielectric Objects" (arXiv 2301.13601).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. The product path (the
 * CUDA library in paper_2301_13601_gb300/) shares no code with it.
 *
 * Every operator is a separate full sweep over the lattice, applied in the
 * order the paper's operator products imply (right-to-left). Arithmetic is
 * IEEE double, compiled with -ffp-contract=off. The only concession to speed
 * is an OpenMP "parallel for" over lattice rows, which does not change any
 * result (every site is computed by exactly one thread, in the same order of
 * operations).
 *
 * State layout: q[c][y][x], c = 0..5, x fastest, periodic in x and y.
 *   Q = (q0..q5) = (n_x E_x, n_y E_y, n_z E_z, B_x, B_y, B_z)   (Eq. 15, mu0 = 1)
 *
 * Readings of the paper taken here (each is pinned by a test):
 *   R1 streaming: S^{+x}_{ij} sets q_c(x) <- q_c(x+1) for c in {i,j}; S^{-x}
 *      sets q_c(x) <- q_c(x-1); the same along y. Operator products act
 *      right-to-left (Eq. 18, Eq. 20, Eq. 23, Eq. 28).
 *   R2 C_Y (Eq. 19): the sin(theta2) entry of row 2 belongs to column 3
 *      (as printed, column 4 makes the matrix non-orthogonal).
 *   R3 V_Y (Eq. 22): row 3 is (0,0,sin b3,cos b3,0,0) (as printed, cos and sin
 *      are swapped, which would not reduce to the identity as b3 -> 0); the
 *      "o" in row 0 is a zero.
 *   R4 external potentials: QLA_POT_PAPER applies V_X, V_Y as printed (with
 *      R3). QLA_POT_UNITARY replaces each printed row pair (target <- cos b
 *      target + t sin b source) by the orthogonal rotation of the same pair by
 *      b/2 (target += t sin(b/2) source, source -= t sin(b/2) target, with
 *      cosines on the diagonal), i.e. the fully unitary variant the paper's
 *      summary names as the next step.
 *   R5 gradients in Eq. 25: central lattice differences
 *      dn/dx = (n[x+1] - n[x-1]) / (2 delta), lattice spacing delta.
 *   R6 interleaved step (Eq. 28): V' (angles halved) after the first eight
 *      and after the last eight operators of U_X, and the same for y.
 *   R7 plain step (Eq. 23): U_X, then U_Y, then V_X, then V_Y.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_POT_PAPER 0
#define ORC_POT_UNITARY 1
#define ORC_SEQ_INTERLEAVED 0
#define ORC_SEQ_PLAIN 1

int orc_version(void) { return 1; }

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static inline size_t plane_of(int Nx, int Ny) { return (size_t)Nx * (size_t)Ny; }
static inline int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }

/* ---------------------------------------------------------------------------
 * Angles. Eq. 24: theta_0 = delta/(4 n_x), theta_1 = delta/(4 n_y),
 * theta_2 = delta/(4 n_z).
 * Eq. 25: beta_0 = delta^2 (dn_y/dx)/n_y^2, beta_1 = delta^2 (dn_x/dy)/n_x^2,
 *         beta_2 = delta^2 (dn_z/dx)/n_z^2, beta_3 = delta^2 (dn_z/dy)/n_z^2,
 * with the physical derivative taken as a central lattice difference over
 * spacing delta (reading R5).
 * theta: 3 planes, beta: 4 planes, each [Ny][Nx].
 * ------------------------------------------------------------------------- */
void orc_angles(int Nx, int Ny, const double *nx, const double *ny, const double *nz,
                double delta, double *theta, double *beta)
{
    const size_t P = plane_of(Nx, Ny);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < Ny; ++y) {
        const int yp = wrap(y + 1, Ny), ym = wrap(y - 1, Ny);
        for (int x = 0; x < Nx; ++x) {
            const int xp = wrap(x + 1, Nx), xm = wrap(x - 1, Nx);
            const size_t i = (size_t)y * Nx + x;
            theta[0 * P + i] = delta / (4.0 * nx[i]);
            theta[1 * P + i] = delta / (4.0 * ny[i]);
            theta[2 * P + i] = delta / (4.0 * nz[i]);
            const double dny_dx = (ny[(size_t)y * Nx + xp] - ny[(size_t)y * Nx + xm]) / (2.0 * delta);
            const double dnx_dy = (nx[(size_t)yp * Nx + x] - nx[(size_t)ym * Nx + x]) / (2.0 * delta);
            const double dnz_dx = (nz[(size_t)y * Nx + xp] - nz[(size_t)y * Nx + xm]) / (2.0 * delta);
            const double dnz_dy = (nz[(size_t)yp * Nx + x] - nz[(size_t)ym * Nx + x]) / (2.0 * delta);
            beta[0 * P + i] = delta * delta * dny_dx / (ny[i] * ny[i]);
            beta[1 * P + i] = delta * delta * dnx_dy / (nx[i] * nx[i]);
            beta[2 * P + i] = delta * delta * dnz_dx / (nz[i] * nz[i]);
            beta[3 * P + i] = delta * delta * dnz_dy / (nz[i] * nz[i]);
        }
    }
}

/* ---------------------------------------------------------------------------
 * Collision C_X (Eq. 17) at every site; dagger != 0 applies its transpose.
 * Rows as printed (c_k = cos theta_k, s_k = sin theta_k):
 *   q0' = q0
 *   q1' = c1 q1 - s1 q5
 *   q2' = c2 q2 - s2 q4
 *   q3' = q3
 *   q4' = s2 q2 + c2 q4
 *   q5' = s1 q1 + c1 q5
 * ------------------------------------------------------------------------- */
void orc_collide_x(int Nx, int Ny, double *q, const double *theta, int dagger)
{
    const size_t P = plane_of(Nx, Ny);
    const double sg = dagger ? -1.0 : 1.0; /* transpose flips the sine signs */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < Ny; ++y) {
        for (int x = 0; x < Nx; ++x) {
            const size_t i = (size_t)y * Nx + x;
            const double t1 = theta[1 * P + i], t2 = theta[2 * P + i];
            const double c1 = cos(t1), s1 = sg * sin(t1);
            const double c2 = cos(t2), s2 = sg * sin(t2);
            const double q1 = q[1 * P + i], q2 = q[2 * P + i], q4 = q[4 * P + i], q5 = q[5 * P + i];
            q[1 * P + i] = c1 * q1 - s1 * q5;
            q[2 * P + i] = c2 * q2 - s2 * q4;
            q[4 * P + i] = s2 * q2 + c2 * q4;
            q[5 * P + i] = s1 * q1 + c1 * q5;
        }
    }
}

/* ---------------------------------------------------------------------------
 * Collision C_Y (Eq. 19, with reading R2) at every site; dagger != 0 applies
 * its transpose. Rows:
 *   q0' = c0 q0 + s0 q5
 *   q1' = q1
 *   q2' = c2 q2 + s2 q3        (printed with s2 in column 4: reading R2)
 *   q3' = -s2 q2 + c2 q3
 *   q4' = q4
 *   q5' = -s0 q0 + c0 q5
 * ------------------------------------------------------------------------- */
void orc_collide_y(int Nx, int Ny, double *q, const double *theta, int dagger)
{
    const size_t P = plane_of(Nx, Ny);
    const double sg = dagger ? -1.0 : 1.0;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < Ny; ++y) {
        for (int x = 0; x < Nx; ++x) {
            const size_t i = (size_t)y * Nx + x;
            const double t0 = theta[0 * P + i], t2 = theta[2 * P + i];
            const double c0 = cos(t0), s0 = sg * sin(t0);
            const double c2 = cos(t2), s2 = sg * sin(t2);
            const double q0 = q[0 * P + i], q2 = q[2 * P + i], q3 = q[3 * P + i], q5 = q[5 * P + i];
            q[0 * P + i] = c0 * q0 + s0 * q5;
            q[2 * P + i] = c2 * q2 + s2 * q3;
            q[3 * P + i] = -s2 * q2 + c2 * q3;
            q[5 * P + i] = -s0 * q0 + c0 * q5;
        }
    }
}

/* ---------------------------------------------------------------------------
 * Streaming S^{dir axis}_{ca cb} (Eq. 18, Eq. 20; reading R1): components ca
 * and cb are moved by one lattice cell, all others are left alone.
 *   dir = +1: q_c(r) <- q_c(r + e_axis);   dir = -1: q_c(r) <- q_c(r - e_axis).
 * axis 0 = x, 1 = y. Periodic.
 * ------------------------------------------------------------------------- */
static void stream_one(int Nx, int Ny, double *p, int axis, int dir)
{
    if (axis == 0) {
#pragma omp parallel for schedule(static)
        for (int y = 0; y < Ny; ++y) {
            double *row = p + (size_t)y * Nx;
            if (dir > 0) {
                const double first = row[0];
                for (int x = 0; x < Nx - 1; ++x) row[x] = row[x + 1];
                row[Nx - 1] = first;
            } else {
                const double last = row[Nx - 1];
                for (int x = Nx - 1; x > 0; --x) row[x] = row[x - 1];
                row[0] = last;
            }
        }
    } else {
        double *tmp = (double *)malloc(sizeof(double) * (size_t)Nx);
        if (dir > 0) {
            memcpy(tmp, p, sizeof(double) * (size_t)Nx);
            for (int y = 0; y < Ny - 1; ++y)
                memcpy(p + (size_t)y * Nx, p + (size_t)(y + 1) * Nx, sizeof(double) * (size_t)Nx);
            memcpy(p + (size_t)(Ny - 1) * Nx, tmp, sizeof(double) * (size_t)Nx);
        } else {
            memcpy(tmp, p + (size_t)(Ny - 1) * Nx, sizeof(double) * (size_t)Nx);
            for (int y = Ny - 1; y > 0; --y)
                memcpy(p + (size_t)y * Nx, p + (size_t)(y - 1) * Nx, sizeof(double) * (size_t)Nx);
            memcpy(p, tmp, sizeof(double) * (size_t)Nx);
        }
        free(tmp);
    }
}

void orc_stream(int Nx, int Ny, double *q, int ca, int cb, int axis, int dir)
{
    const size_t P = plane_of(Nx, Ny);
    stream_one(Nx, Ny, q + (size_t)ca * P, axis, dir);
    stream_one(Nx, Ny, q + (size_t)cb * P, axis, dir);
}

/* ---------------------------------------------------------------------------
 * External potential V_X (Eq. 21) with angles scale*beta (scale = 1 in the
 * plain step Eq. 23, 1/2 in the interleaved step Eq. 28).
 * POT_PAPER rows as printed:
 *   q4' = -sin b2 q2 + cos b2 q4
 *   q5' =  sin b0 q1 + cos b0 q5
 * POT_UNITARY (reading R4): rotate (q4,q2) and (q5,q1) by b/2 so that the
 * target rows receive the same first-order coupling split evenly:
 *   q4' = c q4 - s q2,  q2' = c q2 + s q4   (c,s of b2/2)
 *   q5' = c q5 + s q1,  q1' = c q1 - s q5   (c,s of b0/2)
 * ------------------------------------------------------------------------- */
void orc_potential_x(int Nx, int Ny, double *q, const double *beta, double scale, int mode)
{
    const size_t P = plane_of(Nx, Ny);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < Ny; ++y) {
        for (int x = 0; x < Nx; ++x) {
            const size_t i = (size_t)y * Nx + x;
            const double b0 = scale * beta[0 * P + i], b2 = scale * beta[2 * P + i];
            const double q1 = q[1 * P + i], q2 = q[2 * P + i], q4 = q[4 * P + i], q5 = q[5 * P + i];
            if (mode == ORC_POT_PAPER) {
                q[4 * P + i] = -sin(b2) * q2 + cos(b2) * q4;
                q[5 * P + i] = sin(b0) * q1 + cos(b0) * q5;
            } else {
                const double c2 = cos(0.5 * b2), s2 = sin(0.5 * b2);
                const double c0 = cos(0.5 * b0), s0 = sin(0.5 * b0);
                q[4 * P + i] = c2 * q4 - s2 * q2;
                q[2 * P + i] = c2 * q2 + s2 * q4;
                q[5 * P + i] = c0 * q5 + s0 * q1;
                q[1 * P + i] = c0 * q1 - s0 * q5;
            }
        }
    }
}

/* ---------------------------------------------------------------------------
 * External potential V_Y (Eq. 22, reading R3) with angles scale*beta.
 * POT_PAPER rows:
 *   q3' =  sin b3 q2 + cos b3 q3
 *   q5' = -sin b1 q0 + cos b1 q5
 * POT_UNITARY (reading R4):
 *   q3' = c q3 + s q2,  q2' = c q2 - s q3   (c,s of b3/2)
 *   q5' = c q5 - s q0,  q0' = c q0 + s q5   (c,s of b1/2)
 * ------------------------------------------------------------------------- */
void orc_potential_y(int Nx, int Ny, double *q, const double *beta, double scale, int mode)
{
    const size_t P = plane_of(Nx, Ny);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < Ny; ++y) {
        for (int x = 0; x < Nx; ++x) {
            const size_t i = (size_t)y * Nx + x;
            const double b1 = scale * beta[1 * P + i], b3 = scale * beta[3 * P + i];
            const double q0 = q[0 * P + i], q2 = q[2 * P + i], q3 = q[3 * P + i], q5 = q[5 * P + i];
            if (mode == ORC_POT_PAPER) {
                q[3 * P + i] = sin(b3) * q2 + cos(b3) * q3;
                q[5 * P + i] = -sin(b1) * q0 + cos(b1) * q5;
            } else {
                const double c3 = cos(0.5 * b3), s3 = sin(0.5 * b3);
                const double c1 = cos(0.5 * b1), s1 = sin(0.5 * b1);
                q[3 * P + i] = c3 * q3 + s3 * q2;
                q[2 * P + i] = c3 * q2 - s3 * q3;
                q[5 * P + i] = c1 * q5 - s1 * q0;
                q[0 * P + i] = c1 * q0 + s1 * q5;
            }
        }
    }
}

/* ---------------------------------------------------------------------------
 * Collide-stream sequence along one axis.
 * Eq. 18 printed left to right:
 *   U_X = S+25 C+ S-25 C S-14 C+ S+14 C S-25 C S+25 C+ S+14 C S-14 C+
 * (C+ = dagger). Acting on Q it runs right-to-left:
 *   C+, S-14, C, S+14, C+, S+25, C, S-25, | C, S+14, C+, S-14, C, S-25, C+, S+25
 * Eq. 20 is the same with C_Y, and S03 in place of S14, along y.
 * With mid_v != 0 (Eq. 28) V' is applied at the bar and after the last
 * operator, with angles scaled by vscale.
 * ------------------------------------------------------------------------- */
static void collide(int axis, int Nx, int Ny, double *q, const double *theta, int dagger)
{
    if (axis == 0) orc_collide_x(Nx, Ny, q, theta, dagger);
    else orc_collide_y(Nx, Ny, q, theta, dagger);
}

static void potential(int axis, int Nx, int Ny, double *q, const double *beta, double scale, int mode)
{
    if (axis == 0) orc_potential_x(Nx, Ny, q, beta, scale, mode);
    else orc_potential_y(Nx, Ny, q, beta, scale, mode);
}

void orc_collide_stream(int axis, int Nx, int Ny, double *q, const double *theta,
                        const double *beta, int mid_v, double vscale, int mode)
{
    /* first partner pair streamed along this axis: (1,4) for x, (0,3) for y */
    const int a = axis == 0 ? 1 : 0, b = axis == 0 ? 4 : 3;
    /* ops 1..8 */
    collide(axis, Nx, Ny, q, theta, 1);
    orc_stream(Nx, Ny, q, a, b, axis, -1);
    collide(axis, Nx, Ny, q, theta, 0);
    orc_stream(Nx, Ny, q, a, b, axis, +1);
    collide(axis, Nx, Ny, q, theta, 1);
    orc_stream(Nx, Ny, q, 2, 5, axis, +1);
    collide(axis, Nx, Ny, q, theta, 0);
    orc_stream(Nx, Ny, q, 2, 5, axis, -1);
    if (mid_v) potential(axis, Nx, Ny, q, beta, vscale, mode);
    /* ops 9..16 */
    collide(axis, Nx, Ny, q, theta, 0);
    orc_stream(Nx, Ny, q, a, b, axis, +1);
    collide(axis, Nx, Ny, q, theta, 1);
    orc_stream(Nx, Ny, q, a, b, axis, -1);
    collide(axis, Nx, Ny, q, theta, 0);
    orc_stream(Nx, Ny, q, 2, 5, axis, -1);
    collide(axis, Nx, Ny, q, theta, 1);
    orc_stream(Nx, Ny, q, 2, 5, axis, +1);
    if (mid_v) potential(axis, Nx, Ny, q, beta, vscale, mode);
}

/* ---------------------------------------------------------------------------
 * One time step.
 *   sequence PLAIN (Eq. 23):        Q <- V_Y V_X U_Y U_X Q
 *   sequence INTERLEAVED (Eq. 28):  Q <- [V_Y' U_Y^b V_Y' U_Y^a][V_X' U_X^b V_X' U_X^a] Q
 *                                   with the potential angles halved.
 * ------------------------------------------------------------------------- */
void orc_step(int Nx, int Ny, double *q, const double *theta, const double *beta,
              int sequence, int mode)
{
    if (sequence == ORC_SEQ_PLAIN) {
        orc_collide_stream(0, Nx, Ny, q, theta, beta, 0, 1.0, mode);
        orc_collide_stream(1, Nx, Ny, q, theta, beta, 0, 1.0, mode);
        orc_potential_x(Nx, Ny, q, beta, 1.0, mode);
        orc_potential_y(Nx, Ny, q, beta, 1.0, mode);
    } else {
        orc_collide_stream(0, Nx, Ny, q, theta, beta, 1, 0.5, mode);
        orc_collide_stream(1, Nx, Ny, q, theta, beta, 1, 0.5, mode);
    }
}

void orc_run(int Nx, int Ny, double *q, const double *theta, const double *beta,
             int sequence, int mode, long long nsteps)
{
    for (long long t = 0; t < nsteps; ++t) orc_step(Nx, Ny, q, theta, beta, sequence, mode);
}

/* ---------------------------------------------------------------------------
 * Energy, Eq. 27: E = (1/L^2) \int Q.Q dx dy, i.e. the mean over sites of
 * sum_c q_c^2. Neumaier-compensated summation, serial and in site order.
 * ------------------------------------------------------------------------- */
static void neumaier_add(double *sum, double *comp, double v)
{
    const double t = *sum + v;
    if (fabs(*sum) >= fabs(v)) *comp += (*sum - t) + v;
    else *comp += (v - t) + *sum;
    *sum = t;
}

double orc_energy(int Nx, int Ny, const double *q)
{
    const size_t P = plane_of(Nx, Ny);
    double s = 0.0, c = 0.0;
    for (size_t i = 0; i < P; ++i) {
        double e = 0.0;
        for (int k = 0; k < 6; ++k) e += q[(size_t)k * P + i] * q[(size_t)k * P + i];
        neumaier_add(&s, &c, e);
    }
    return (s + c) / (double)P;
}

/* ---------------------------------------------------------------------------
 * Divergence of B (the diagnostic behind the paper's max div B/|B| < 1e-3
 * statement in Sec. 4.1), in lattice units with central differences at the
 * sites: div = (B_x[x+1]-B_x[x-1])/2 + (B_y[y+1]-B_y[y-1])/2, B_x = q3,
 * B_y = q4 (B_z does not vary in z for 2D fields).
 * out[0] = sum div^2, out[1] = max |div|, out[2] = max |B| = max sqrt(q3^2+q4^2+q5^2).
 * ------------------------------------------------------------------------- */
void orc_divB(int Nx, int Ny, const double *q, double *out)
{
    const size_t P = plane_of(Nx, Ny);
    double s = 0.0, c = 0.0, mdiv = 0.0, mb = 0.0;
    for (int y = 0; y < Ny; ++y) {
        const int yp = wrap(y + 1, Ny), ym = wrap(y - 1, Ny);
        for (int x = 0; x < Nx; ++x) {
            const int xp = wrap(x + 1, Nx), xm = wrap(x - 1, Nx);
            const size_t i = (size_t)y * Nx + x;
            const double d = 0.5 * (q[3 * P + (size_t)y * Nx + xp] - q[3 * P + (size_t)y * Nx + xm]) +
                             0.5 * (q[4 * P + (size_t)yp * Nx + x] - q[4 * P + (size_t)ym * Nx + x]);
            neumaier_add(&s, &c, d * d);
            if (fabs(d) > mdiv) mdiv = fabs(d);
            const double b = sqrt(q[3 * P + i] * q[3 * P + i] + q[4 * P + i] * q[4 * P + i] +
                                  q[5 * P + i] * q[5 * P + i]);
            if (b > mb) mb = b;
        }
    }
    out[0] = s + c;
    out[1] = mdiv;
    out[2] = mb;
}

/* ---------------------------------------------------------------------------
 * Divergence of D (Sec. 4.2: with the E_y polarisation the QLA generates an
 * E_x field so that div D = 0), in lattice units with central differences at
 * the sites. The dielectric tensor is diagonal with eps_i = n_i^2, so with
 * q0 = n_x E_x, q1 = n_y E_y, q2 = n_z E_z (Eq. 15):
 *   D_x = n_x q0,  D_y = n_y q1,  D_z = n_z q2 (no z dependence in 2D),
 *   div = (D_x[x+1]-D_x[x-1])/2 + (D_y[y+1]-D_y[y-1])/2.
 * out[0] = sum div^2, out[1] = max |div|, out[2] = max |D|.
 * ------------------------------------------------------------------------- */
void orc_divD(int Nx, int Ny, const double *q, const double *nx, const double *ny, const double *nz, double *out)
{
    const size_t P = plane_of(Nx, Ny);
    double s = 0.0, c = 0.0, mdiv = 0.0, md = 0.0;
    for (int y = 0; y < Ny; ++y) {
        const int yp = wrap(y + 1, Ny), ym = wrap(y - 1, Ny);
        for (int x = 0; x < Nx; ++x) {
            const int xp = wrap(x + 1, Nx), xm = wrap(x - 1, Nx);
            const size_t i = (size_t)y * Nx + x;
            const size_t ixp = (size_t)y * Nx + xp, ixm = (size_t)y * Nx + xm;
            const size_t iyp = (size_t)yp * Nx + x, iym = (size_t)ym * Nx + x;
            const double d = 0.5 * (nx[ixp] * q[0 * P + ixp] - nx[ixm] * q[0 * P + ixm]) +
                             0.5 * (ny[iyp] * q[1 * P + iyp] - ny[iym] * q[1 * P + iym]);
            neumaier_add(&s, &c, d * d);
            if (fabs(d) > mdiv) mdiv = fabs(d);
            const double dx = nx[i] * q[0 * P + i], dy = ny[i] * q[1 * P + i], dz = nz[i] * q[2 * P + i];
            const double dm = sqrt(dx * dx + dy * dy + dz * dz);
            if (dm > md) md = dm;
        }
    }
    out[0] = s + c;
    out[1] = mdiv;
    out[2] = md;
}

/* ---------------------------------------------------------------------------
 * Initial 1D Gaussian pulse travelling in +x (Sec. 2.2 energy discussion and
 * Sec. 4: a 1D pulse propagating in x). g(x) = amp exp(-d^2/(2 sigma^2)) with
 * d the periodic minimum-image distance x - x0; uniform in y.
 *   pol 0 (E_z): q2 = g, q4 = -g   (B_y paired for +x travel, from Eq. 16)
 *   pol 1 (E_y): q1 = g, q5 = +g   (B_z paired for +x travel, from Eq. 16)
 * All other components are zero.
 * ------------------------------------------------------------------------- */
void orc_init_pulse(int Nx, int Ny, double *q, int pol, double x0, double sigma, double amp)
{
    const size_t P = plane_of(Nx, Ny);
    memset(q, 0, sizeof(double) * 6 * P);
    for (int x = 0; x < Nx; ++x) {
        double d = (double)x - x0;
        d -= (double)Nx * floor(d / (double)Nx + 0.5);
        const double g = amp * exp(-d * d / (2.0 * sigma * sigma));
        for (int y = 0; y < Ny; ++y) {
            const size_t i = (size_t)y * Nx + x;
            if (pol == 0) {
                q[2 * P + i] = g;
                q[4 * P + i] = -g;
            } else {
                q[1 * P + i] = g;
                q[5 * P + i] = g;
            }
        }
    }
}

/* ---------------------------------------------------------------------------
 * Brute-force Yee FDTD comparator for the continuum equations the QLA is meant
 * to recover (Eq. 16 in the basis E, B with eps_i = n_i^2, mu0 = 1).
 * Periodic Nx x Ny grid of spacing h, time step dt, leapfrog.
 * Staggering (cell indices i = x, j = y):
 *   E_z(i,j)        B_x(i,j+1/2)    B_y(i+1/2,j)
 *   E_x(i+1/2,j)    E_y(i,j+1/2)    B_z(i+1/2,j+1/2)
 * Arrays are [Ny][Nx]; entry (j,i) holds the value at the staggered point
 * listed above. eps: 3 planes (eps_x at E_x points, eps_y at E_y points,
 * eps_z at E_z points). E: (E_x, E_y, E_z), B: (B_x, B_y, B_z), all at t = 0
 * on entry and at t = nsteps dt on return.
 *   dB/dt = -curl E,   eps dE/dt = curl B.
 * ------------------------------------------------------------------------- */
static void yee_update_B(int Nx, int Ny, const double *E, double *B, double k)
{
    const size_t P = plane_of(Nx, Ny);
    const double *Ex = E, *Ey = E + P, *Ez = E + 2 * P;
    double *Bx = B, *By = B + P, *Bz = B + 2 * P;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < Ny; ++j) {
        const int jp = wrap(j + 1, Ny);
        for (int i = 0; i < Nx; ++i) {
            const int ip = wrap(i + 1, Nx);
            const size_t c = (size_t)j * Nx + i;
            /* dBx/dt = -dEz/dy at (i, j+1/2) */
            Bx[c] -= k * (Ez[(size_t)jp * Nx + i] - Ez[c]);
            /* dBy/dt = +dEz/dx at (i+1/2, j) */
            By[c] += k * (Ez[(size_t)j * Nx + ip] - Ez[c]);
            /* dBz/dt = dEx/dy - dEy/dx at (i+1/2, j+1/2) */
            Bz[c] += k * ((Ex[(size_t)jp * Nx + i] - Ex[c]) - (Ey[(size_t)j * Nx + ip] - Ey[c]));
        }
    }
}

static void yee_update_E(int Nx, int Ny, double *E, const double *B, const double *eps, double k)
{
    const size_t P = plane_of(Nx, Ny);
    double *Ex = E, *Ey = E + P, *Ez = E + 2 * P;
    const double *Bx = B, *By = B + P, *Bz = B + 2 * P;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < Ny; ++j) {
        const int jm = wrap(j - 1, Ny);
        for (int i = 0; i < Nx; ++i) {
            const int im = wrap(i - 1, Nx);
            const size_t c = (size_t)j * Nx + i;
            /* eps_z dEz/dt = dBy/dx - dBx/dy at (i, j) */
            Ez[c] += k / eps[2 * P + c] *
                     ((By[c] - By[(size_t)j * Nx + im]) - (Bx[c] - Bx[(size_t)jm * Nx + i]));
            /* eps_x dEx/dt = dBz/dy at (i+1/2, j) */
            Ex[c] += k / eps[0 * P + c] * (Bz[c] - Bz[(size_t)jm * Nx + i]);
            /* eps_y dEy/dt = -dBz/dx at (i, j+1/2) */
            Ey[c] -= k / eps[1 * P + c] * (Bz[c] - Bz[(size_t)j * Nx + im]);
        }
    }
}

void orc_yee_run(int Nx, int Ny, double h, double dt, long long nsteps, const double *eps,
                 double *E, double *B)
{
    const double k = dt / h;
    if (nsteps <= 0) return;
    yee_update_B(Nx, Ny, E, B, 0.5 * k); /* B to t = dt/2 */
    for (long long n = 1; n <= nsteps; ++n) {
        yee_update_E(Nx, Ny, E, B, eps, k);
        yee_update_B(Nx, Ny, E, B, n < nsteps ? k : 0.5 * k);
    }
}
