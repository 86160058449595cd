/*
 * fgs4d_oracle.c -- plain, slow, double-precision CPU oracle for the 4D
 * Gaussian Splatting rendering routine (Yang et al., "Real-time
 * Photorealistic Dynamic Scene Representation and Rendering with 4D Gaussian
 * Splatting", ICLR 2024) and for its adjoint.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file.
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * load it.  It shares no code, header, table or constant with the CUDA path.
 *
 * What it computes, step by step, in the paper's order:
 *   O1  activations: s = exp(log s), alpha = sigmoid(logit), unit quaternions
 *   O2  4D rotation R = L(q_l) R(q_r) exactly as printed (Eq. 8) and the
 *       covariance Sigma = R S S^T R^T (Eq. 7)
 *   O3  marginal p(t) = exp(-1/2 (t-mu_t)^2 / Sigma_44) (Eq. 10, read as the
 *       unnormalised Gaussian of Eq. 1) and the p(t) < 0.05 filter (Sec. 4.2)
 *   O4  conditional 3D Gaussian by Schur complement (Eq. 9)
 *   O5  4D spherindrical-harmonic colour (Eq. 11)
 *   O6  EWA splatting of the conditional Gaussian (Eq. 3, Eq. 4)
 *   O7  time-aware front-to-back compositing of every pixel over ALL splats
 *       sorted by (depth, index) (Eq. 6), i.e. the definition, no tiling
 *   O9  the hand-derived reverse-mode gradient of O7 -> O1
 *
 * Readings of points the paper leaves open (kept identical on the GPU side,
 * each one an explicit option or documented constant):
 *   R1  p(t) and p(u,v|t) are unnormalised (peak value 1)
 *   R2  the product in Eq. 2 uses p_j (Eq. 5/6), not p_i
 *   R4  alpha = min(alpha_max, alpha_eff * G); skip when alpha < alpha_min
 *   R5  stop before splat i when T * (1 - alpha_i) < T_min (i not added)
 *   R6  skip when the exponent is positive (round-off guard)
 *   R7  support radius r = sqrt(2 ln(alpha_eff/alpha_min) lambda_max)
 *   R8  ties in depth are broken by ascending Gaussian index
 *   R9  4DSH uses cos(2 pi n dt / T), n = 0..K, dt = t - mu_t
 *   R11 real orthonormal SH (Condon-Shortley phase), colour = max(sum+0.5, 0),
 *       view direction from the camera centre to the conditional mean
 *   R13 OpenCV pinhole (+z forward); optional clamp of x/z, y/z inside J
 *   R14 isotropic dilation delta added to the 2D covariance
 *   R15 pixel (i, j) is sampled at image coordinates (i, j)
 *
 * Pixel flags (out parameter of orc_render): a pixel is flagged when one of
 * the discrete decisions taken for it lies within a relative margin of its
 * threshold, where a single-precision evaluation may legitimately decide the
 * other way: bit 0 = the image value may differ (alpha_min skip, early
 * termination, depth order, a borderline Gaussian-level cull), bit 1 = only
 * the gradient may differ (alpha_max clamp, colour clamp, depth near-tie).  Bits 2..5 name
 * the cause of bit 0: depth order, early termination, alpha_min skip,
 * Gaussian-level cull.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_API __attribute__((visibility("default")))

/* relative margins used only for pixel flags (see header comment) */
#define ORC_ETA_ALPHA 1e-4
#define ORC_ETA_T 2e-3
#define ORC_ETA_DEPTH 2e-6
#define ORC_ETA_P 1e-4
#define ORC_ETA_NEAR 1e-4

typedef struct {
    int64_t n;         /* number of Gaussians */
    int sh_degree;     /* L */
    int n_freq;        /* K: Fourier orders n = 0..K */
    double period;     /* T of Eq. 11 */
    const double *mu;     /* [4][n]  (x, y, z, t) */
    const double *log_s;  /* [4][n] */
    const double *ql;     /* [4][n]  (a, b, c, d) scalar first */
    const double *qr;     /* [4][n]  (p, q, r, s) scalar first */
    const double *logit;  /* [n] */
    const double *shs;    /* [3*(L+1)^2*(K+1)][n], row = (f*(L+1)^2 + j)*3 + ch */
} orc_gaussians;

typedef struct {
    double viewmat[12];  /* row-major 3x4 [W | tau], world -> camera */
    double fx, fy, cx, cy;
    int width, height;
    double t;
    double bg[3];
} orc_view;

typedef struct {
    double p_min;      /* temporal filter threshold (0.05) */
    double near_z;     /* near plane (0.2) */
    double alpha_min;  /* 1/255 */
    double alpha_max;  /* 0.99 */
    double T_min;      /* 1e-4 */
    double dilation;   /* delta added to Sigma_2d diagonal */
    double clamp_fov;  /* 0 = off; else x/z limited to clamp_fov * W/(2 fx) */
} orc_options;

typedef struct {
    int visible;       /* 1 when the splat can contribute */
    int cull;          /* 0 visible, 1 p<p_min, 2 near, 3 alpha_eff<alpha_min, 4 det<=0 */
    int borderline;    /* a Gaussian-level decision is within its margin */
    double p_t;
    double mu3[3];
    double Sigma3[9];
    double xc[3];
    double u, v, depth;
    double cov2d[3];   /* (S00, S01, S11) */
    double conic[3];   /* (a, b, c) = inverse of cov2d */
    double alpha, alpha_eff;
    double color[3], color_raw[3];
    double radius;     /* exact R7 bound, no margin */
} orc_splat;

typedef struct {
    double *mu, *log_s, *ql, *qr, *logit, *shs;  /* same layout as inputs, accumulated */
} orc_grads;

/* ------------------------------------------------------------------ */
/* small dense helpers (row-major)                                      */
/* ------------------------------------------------------------------ */
static void matmul(const double *A, const double *B, double *C, int n, int k, int m) {
    for (int i = 0; i < n; i++)
        for (int j = 0; j < m; j++) {
            double acc = 0.0;
            for (int l = 0; l < k; l++) acc += A[i * k + l] * B[l * m + j];
            C[i * m + j] = acc;
        }
}
static void transpose(const double *A, double *At, int n, int m) {
    for (int i = 0; i < n; i++)
        for (int j = 0; j < m; j++) At[j * n + i] = A[i * m + j];
}

/* ------------------------------------------------------------------ */
/* O1 + O2: Eq. 7 and Eq. 8                                             */
/* ------------------------------------------------------------------ */

/* Left isoclinic matrix L(q_l) of Eq. 8, q = (a, b, c, d). */
ORC_API void orc_quat_left(const double *q, double *L) {
    const double a = q[0], b = q[1], c = q[2], d = q[3];
    const double M[16] = {a, -b, -c, -d,
                          b,  a, -d,  c,
                          c,  d,  a, -b,
                          d, -c,  b,  a};
    memcpy(L, M, sizeof(M));
}

/* Right isoclinic matrix R(q_r) of Eq. 8, q = (p, q, r, s). */
ORC_API void orc_quat_right(const double *q, double *R) {
    const double p = q[0], qq = q[1], r = q[2], s = q[3];
    const double M[16] = {p, -qq, -r, -s,
                          qq,  p,  s, -r,
                          r,  -s,  p, qq,
                          s,   r, -qq, p};
    memcpy(R, M, sizeof(M));
}

static void normalize4(const double *q, double *qn, double *norm) {
    double n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    double n = sqrt(n2);
    *norm = n;
    for (int i = 0; i < 4; i++) qn[i] = q[i] / n;
}

/* R = L(q_l / |q_l|) R(q_r / |q_r|)  (Eq. 8). */
ORC_API void orc_rotation4(const double *ql, const double *qr, double *R) {
    double qln[4], qrn[4], nl, nr, L[16], Rr[16];
    normalize4(ql, qln, &nl);
    normalize4(qr, qrn, &nr);
    orc_quat_left(qln, L);
    orc_quat_right(qrn, Rr);
    matmul(L, Rr, R, 4, 4, 4);
}

/* Sigma = R S S^T R^T with S = diag(exp(log_s))  (Eq. 7). */
ORC_API void orc_covariance4(const double *log_s, const double *ql, const double *qr, double *Sigma) {
    double R[16], M[16], Mt[16];
    orc_rotation4(ql, qr, R);
    for (int i = 0; i < 4; i++)
        for (int k = 0; k < 4; k++) M[i * 4 + k] = R[i * 4 + k] * exp(log_s[k]);
    transpose(M, Mt, 4, 4);
    matmul(M, Mt, Sigma, 4, 4, 4);
}

/* ------------------------------------------------------------------ */
/* O3 + O4: Eq. 9 and Eq. 10                                            */
/* ------------------------------------------------------------------ */
ORC_API void orc_condition(const double *mu, const double *Sigma, double t,
                           double *mu3, double *Sigma3, double *p_t) {
    const double s44 = Sigma[15];
    const double dt = t - mu[3];
    for (int i = 0; i < 3; i++) mu3[i] = mu[i] + Sigma[i * 4 + 3] / s44 * dt;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            Sigma3[i * 3 + j] = Sigma[i * 4 + j] - Sigma[i * 4 + 3] / s44 * Sigma[3 * 4 + j];
    *p_t = exp(-0.5 * dt * dt / s44);
}

/* ------------------------------------------------------------------ */
/* O5: real spherical harmonics from their closed form, Eq. 11          */
/*                                                                      */
/* Y_l^0  = K_l^0 P_l(z)                                                */
/* Y_l^m  = sqrt2 K_l^m (-1)^m P_l^(m)(z) Re((x+iy)^m)   (m > 0)        */
/* Y_l^-m = sqrt2 K_l^m (-1)^m P_l^(m)(z) Im((x+iy)^m)   (m > 0)        */
/* with K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), P_l^(m) the m-th     */
/* derivative of the Legendre polynomial; on the unit sphere this is   */
/* the associated Legendre function with Condon-Shortley phase.  The    */
/* index of (l, m) is j = l^2 + l + m.                                  */
/* ------------------------------------------------------------------ */
static double factorial(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; i++) f *= i;
    return f;
}
static double binom(int n, int k) { return factorial(n) / (factorial(k) * factorial(n - k)); }

/* coefficients c[0..l] of P_l(z) = sum c[k] z^k (Rodrigues' formula expanded) */
static void legendre_coeffs(int l, double *c) {
    for (int k = 0; k <= l; k++) c[k] = 0.0;
    for (int k = 0; 2 * k <= l; k++)
        c[l - 2 * k] = pow(-1.0, k) * binom(l, k) * binom(2 * l - 2 * k, l) / pow(2.0, l);
}
/* value of the m-th derivative of the polynomial with coefficients c (degree l) */
static double poly_deriv_eval(const double *c, int l, int m, double z) {
    double acc = 0.0;
    for (int k = m; k <= l; k++) {
        double fall = 1.0;
        for (int i = 0; i < m; i++) fall *= (double)(k - i);
        acc += c[k] * fall * pow(z, k - m);
    }
    return acc;
}

/* Y[(L+1)^2] at the point d (any 3-vector, evaluated as a polynomial);
   dY[3*(L+1)^2] (optional) = gradient of each polynomial w.r.t. (x, y, z). */
ORC_API void orc_sh_basis(int L, const double *d, double *Y, double *dY) {
    const double x = d[0], y = d[1], z = d[2];
    /* A_m = Re((x+iy)^m), B_m = Im((x+iy)^m) */
    double A[16], B[16];
    A[0] = 1.0; B[0] = 0.0;
    for (int m = 1; m <= L; m++) {
        A[m] = A[m - 1] * x - B[m - 1] * y;
        B[m] = A[m - 1] * y + B[m - 1] * x;
    }
    for (int l = 0; l <= L; l++) {
        double c[16];
        legendre_coeffs(l, c);
        for (int m = 0; m <= l; m++) {
            double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - m) / factorial(l + m));
            double D = poly_deriv_eval(c, l, m, z);
            double Dz = poly_deriv_eval(c, l, m + 1, z);
            if (m == 0) {
                int j = l * l + l;
                Y[j] = K * D;
                if (dY) {
                    dY[3 * j + 0] = 0.0;
                    dY[3 * j + 1] = 0.0;
                    dY[3 * j + 2] = K * Dz;
                }
            } else {
                double f = sqrt(2.0) * K * ((m % 2) ? -1.0 : 1.0);
                int jp = l * l + l + m, jn = l * l + l - m;
                Y[jp] = f * D * A[m];
                Y[jn] = f * D * B[m];
                if (dY) {
                    /* d/dx A_m = m A_{m-1}, d/dy A_m = -m B_{m-1};
                       d/dx B_m = m B_{m-1}, d/dy B_m =  m A_{m-1} */
                    dY[3 * jp + 0] = f * D * m * A[m - 1];
                    dY[3 * jp + 1] = f * D * (-m) * B[m - 1];
                    dY[3 * jp + 2] = f * Dz * A[m];
                    dY[3 * jn + 0] = f * D * m * B[m - 1];
                    dY[3 * jn + 1] = f * D * m * A[m - 1];
                    dY[3 * jn + 2] = f * Dz * B[m];
                }
            }
        }
    }
}

static int n_sh(const orc_gaussians *G) { return (G->sh_degree + 1) * (G->sh_degree + 1); }
static int n_coef(const orc_gaussians *G) { return n_sh(G) * (G->n_freq + 1); }

static double gparam(const double *arr, int row, int64_t g, int64_t n) { return arr[(int64_t)row * n + g]; }

/* camera centre C = -W^T tau */
static void camera_center(const orc_view *V, double *C) {
    for (int i = 0; i < 3; i++) {
        C[i] = 0.0;
        for (int k = 0; k < 3; k++) C[i] -= V->viewmat[k * 4 + i] * V->viewmat[k * 4 + 3];
    }
}

/* raw colour (before +0.5 and clamp): sum_n cos(2 pi n dt / T) sum_j k Y_j(d) */
static void sh4d_color(const orc_gaussians *G, int64_t g, const double *dir, double dt, double *raw) {
    const int nb = n_sh(G);
    double Y[64];
    orc_sh_basis(G->sh_degree, dir, Y, NULL);
    for (int ch = 0; ch < 3; ch++) {
        double acc = 0.0;
        for (int f = 0; f <= G->n_freq; f++) {
            double cf = cos(2.0 * M_PI * f * dt / G->period);
            for (int j = 0; j < nb; j++) acc += cf * gparam(G->shs, (f * nb + j) * 3 + ch, g, G->n) * Y[j];
        }
        raw[ch] = acc;
    }
}

/* ------------------------------------------------------------------ */
/* O1..O6 for one Gaussian and one view                                 */
/* ------------------------------------------------------------------ */
static void jacobian(const orc_view *V, const orc_options *O, const double *xc, double *J,
                     int *clamped_x, int *clamped_y) {
    const double X = xc[0], Y = xc[1], Z = xc[2];
    double tx = X / Z, ty = Y / Z;
    *clamped_x = 0;
    *clamped_y = 0;
    if (O->clamp_fov > 0.0) {
        double limx = O->clamp_fov * 0.5 * V->width / V->fx;
        double limy = O->clamp_fov * 0.5 * V->height / V->fy;
        if (tx < -limx) { tx = -limx; *clamped_x = 1; }
        if (tx > limx) { tx = limx; *clamped_x = 1; }
        if (ty < -limy) { ty = -limy; *clamped_y = 1; }
        if (ty > limy) { ty = limy; *clamped_y = 1; }
    }
    J[0] = V->fx / Z; J[1] = 0.0;       J[2] = -V->fx * tx / Z;
    J[3] = 0.0;       J[4] = V->fy / Z; J[5] = -V->fy * ty / Z;
}

ORC_API int orc_project(const orc_gaussians *G, int64_t g, const orc_view *V, const orc_options *O,
                        orc_splat *S) {
    memset(S, 0, sizeof(*S));
    const int64_t n = G->n;
    double mu[4], ls[4], ql[4], qr[4];
    for (int i = 0; i < 4; i++) {
        mu[i] = gparam(G->mu, i, g, n);
        ls[i] = gparam(G->log_s, i, g, n);
        ql[i] = gparam(G->ql, i, g, n);
        qr[i] = gparam(G->qr, i, g, n);
    }
    /* O1 */
    const double alpha = 1.0 / (1.0 + exp(-G->logit[g]));
    /* O2 */
    double Sigma[16];
    orc_covariance4(ls, ql, qr, Sigma);
    /* O3 + O4 */
    orc_condition(mu, Sigma, V->t, S->mu3, S->Sigma3, &S->p_t);
    S->alpha = alpha;
    S->alpha_eff = alpha * S->p_t;
    if (fabs(S->p_t - O->p_min) <= ORC_ETA_P * O->p_min) S->borderline = 1;
    if (S->p_t < O->p_min) { S->cull = 1; }
    /* O6 (camera part) */
    for (int i = 0; i < 3; i++) {
        S->xc[i] = V->viewmat[i * 4 + 3];
        for (int k = 0; k < 3; k++) S->xc[i] += V->viewmat[i * 4 + k] * S->mu3[k];
    }
    const double Z = S->xc[2];
    if (fabs(Z - O->near_z) <= ORC_ETA_NEAR * O->near_z) S->borderline = 1;
    if (S->cull == 0 && Z < O->near_z) S->cull = 2;
    if (Z <= 1e-9) { /* behind the camera: no projection is defined */
        if (S->cull == 0) S->cull = 2;
        return S->visible = 0;
    }
    S->depth = Z;
    S->u = V->fx * S->xc[0] / Z + V->cx;
    S->v = V->fy * S->xc[1] / Z + V->cy;
    double J[6], W[9], T[6], Tt[6], tmp[6], C2[4];
    int cx_, cy_;
    jacobian(V, O, S->xc, J, &cx_, &cy_);
    for (int i = 0; i < 3; i++)
        for (int k = 0; k < 3; k++) W[i * 3 + k] = V->viewmat[i * 4 + k];
    matmul(J, W, T, 2, 3, 3);             /* T = J W */
    matmul(T, S->Sigma3, tmp, 2, 3, 3);   /* T Sigma3 */
    transpose(T, Tt, 2, 3);
    matmul(tmp, Tt, C2, 2, 3, 2);         /* Eq. 4: J W Sigma3 W^T J^T */
    S->cov2d[0] = C2[0] + O->dilation;
    S->cov2d[1] = C2[1];
    S->cov2d[2] = C2[3] + O->dilation;
    const double det = S->cov2d[0] * S->cov2d[2] - S->cov2d[1] * S->cov2d[1];
    if (det <= 0.0) {
        if (S->cull == 0) S->cull = 4;
        return S->visible = 0;
    }
    S->conic[0] = S->cov2d[2] / det;
    S->conic[1] = -S->cov2d[1] / det;
    S->conic[2] = S->cov2d[0] / det;
    if (fabs(S->alpha_eff - O->alpha_min) <= ORC_ETA_ALPHA * O->alpha_min) S->borderline = 1;
    if (S->cull == 0 && S->alpha_eff < O->alpha_min) S->cull = 3;
    /* R7 support radius */
    const double mid = 0.5 * (S->cov2d[0] + S->cov2d[2]);
    const double lmax = mid + sqrt(fmax(mid * mid - det, 0.0));
    const double lnr = log(S->alpha_eff / O->alpha_min);
    S->radius = lnr > 0.0 ? sqrt(2.0 * lnr * lmax) : 0.0;
    /* O5: colour seen from the camera centre towards the conditional mean */
    double Cc[3], dir[3];
    camera_center(V, Cc);
    double nrm = 0.0;
    for (int i = 0; i < 3; i++) { dir[i] = S->mu3[i] - Cc[i]; nrm += dir[i] * dir[i]; }
    nrm = sqrt(nrm);
    for (int i = 0; i < 3; i++) dir[i] /= nrm;
    sh4d_color(G, g, dir, V->t - mu[3], S->color_raw);
    for (int ch = 0; ch < 3; ch++) S->color[ch] = fmax(S->color_raw[ch] + 0.5, 0.0);
    S->visible = (S->cull == 0);
    return S->visible;
}

/* ------------------------------------------------------------------ */
/* O7: the definition of Eq. 6, per pixel over all splats               */
/* ------------------------------------------------------------------ */
typedef struct { double depth; int64_t idx; } depth_key;
static int cmp_depth(const void *a, const void *b) {
    const depth_key *x = (const depth_key *)a, *y = (const depth_key *)b;
    if (x->depth < y->depth) return -1;
    if (x->depth > y->depth) return 1;
    return (x->idx < y->idx) ? -1 : (x->idx > y->idx);
}

/* splats that can matter for some pixel: visible ones, plus culled ones whose
   cull decision is borderline (those only raise flags) */
static int64_t sorted_candidates(const orc_gaussians *G, const orc_view *V, const orc_options *O,
                                 orc_splat *S, int64_t **order_out) {
    depth_key *keys = (depth_key *)malloc(sizeof(depth_key) * (G->n > 0 ? G->n : 1));
    int64_t m = 0;
    for (int64_t g = 0; g < G->n; g++) {
        orc_project(G, g, V, O, &S[g]);
        int cand = S[g].visible || (S[g].borderline && S[g].depth > 0.0 &&
                                    (S[g].cov2d[0] * S[g].cov2d[2] - S[g].cov2d[1] * S[g].cov2d[1]) > 0.0);
        if (cand) { keys[m].depth = S[g].depth; keys[m].idx = g; m++; }
    }
    qsort(keys, (size_t)m, sizeof(depth_key), cmp_depth);
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (m > 0 ? m : 1));
    for (int64_t i = 0; i < m; i++) order[i] = keys[i].idx;
    free(keys);
    *order_out = order;
    return m;
}

typedef struct {
    int64_t g;
    double alpha, araw, Gexp, T, dx, dy;
    int clamped;
} contrib;

/* Walks one pixel front to back.  Fills the contributor list (if given),
   returns the number of contributors; writes colour, final T and flags.

   amb (optional, two doubles) bounds how far a valid single-precision
   evaluation may land from this result, summed over the flagged decisions:
   amb[0] for the colour, amb[1] for the final transmittance.  cmax bounds
   every colour component (splats and background).  A splat included or
   skipped the other way moves the pixel by at most T a (|c| + cmax) and T by
   T a; two adjacent splats blended in the other order move it by exactly
   T a_1 a_2 (c_1 - c_2) and leave T unchanged; stopping one splat earlier or
   later moves it by at most T (a (|c| + cmax) + cmax) and T by T. */
static int pixel_walk(const orc_splat *S, const int64_t *order, int64_t m, const orc_options *O,
                      const orc_view *V, double px, double py, int prefilter, double *C, double *T_out,
                      uint8_t *flag, contrib *list, uint64_t *hash, double *amb, double cmax) {
    double T = 1.0;
    uint64_t hsh = 1469598103934665603ull; /* order-sensitive hash of the contributor sequence */
    C[0] = C[1] = C[2] = 0.0;
    int nc = 0;
    uint8_t f = 0;
    /* previous relevant splat, for the depth-order check */
    double last_rel_depth = -1.0, last_alpha = 0.0, last_T = 1.0;
    const double *last_color = NULL;
    double amb_c = 0.0, amb_t = 0.0;
    for (int64_t k = 0; k < m; k++) {
        const orc_splat *s = &S[order[k]];
        const double dx = px - s->u, dy = py - s->v;
        if (prefilter) {
            double r = s->radius * (1.0 + 1e-3) + 1.0;
            if (dx * dx + dy * dy > r * r) continue;
        }
        const double power = -0.5 * (s->conic[0] * dx * dx + s->conic[2] * dy * dy) - s->conic[1] * dx * dy;
        const double Gexp = exp(power);
        const double araw = s->alpha_eff * Gexp;
        const int relevant = araw >= O->alpha_min * (1.0 - ORC_ETA_ALPHA);
        double cs = 0.0;
        for (int ch = 0; ch < 3; ch++) cs = fmax(cs, fabs(s->color[ch]));
        if (relevant) {
            const double a_cl = araw < O->alpha_max ? araw : O->alpha_max;
            int flip = 0;
            if (s->borderline) { f |= 1 | 32; flip = 1; }
            if (fabs(araw - O->alpha_min) <= ORC_ETA_ALPHA * O->alpha_min) { f |= 1 | 16; flip = 1; }
            if (flip) {
                amb_c += T * a_cl * (cs + cmax);
                amb_t += T * a_cl;
            }
            if (last_rel_depth >= 0.0 && fabs(s->depth - last_rel_depth) <= ORC_ETA_DEPTH * s->depth) {
                double dc = 0.0;
                for (int ch = 0; ch < 3; ch++) dc = fmax(dc, fabs(s->color[ch] - last_color[ch]));
                const double d = last_T * a_cl * last_alpha * dc;
                f |= 2;
                if (d > 1e-5) f |= 1 | 4; /* below 1e-5 the image cannot tell */
                amb_c += d;
            }
            last_rel_depth = s->depth;
            last_alpha = a_cl;
            last_color = s->color;
            last_T = T;
        }
        if (!s->visible) continue; /* borderline-culled: flags only */
        if (power > 0.0) continue;  /* R6 */
        double alpha = araw < O->alpha_max ? araw : O->alpha_max;  /* R4 */
        if (alpha < O->alpha_min) continue;
        if (fabs(araw - O->alpha_max) <= ORC_ETA_ALPHA * O->alpha_max) f |= 2;
        const double Tn = T * (1.0 - alpha);
        if (fabs(Tn - O->T_min) <= ORC_ETA_T * O->T_min) {
            f |= 1 | 8;
            amb_c += T * (alpha * (cs + cmax) + cmax);
            amb_t += T;
        }
        if (Tn < O->T_min) break;  /* R5 */
        for (int ch = 0; ch < 3; ch++) {
            C[ch] += s->color[ch] * alpha * T;
            if (fabs(s->color_raw[ch] + 0.5) <= 1e-6) f |= 2;
        }
        if (list) {
            contrib *c = &list[nc];
            c->g = order[k]; c->alpha = alpha; c->araw = araw; c->Gexp = Gexp; c->T = T;
            c->dx = dx; c->dy = dy; c->clamped = araw > O->alpha_max;
        }
        nc++;
        hsh = hsh * 1099511628211ull + (uint64_t)(order[k] + 1);
        T = Tn;
    }
    for (int ch = 0; ch < 3; ch++) C[ch] += T * V->bg[ch];
    *T_out = T;
    if (flag) *flag = f;
    if (hash) *hash = hsh;
    if (amb) {
        amb[0] = amb_c;
        amb[1] = amb_t;
    }
    return nc;
}

/* largest colour component of the candidates and the background */
static double max_color(const orc_splat *S, const int64_t *order, int64_t m, const orc_view *V) {
    double c = 0.0;
    for (int ch = 0; ch < 3; ch++) c = fmax(c, fabs(V->bg[ch]));
    for (int64_t k = 0; k < m; k++)
        for (int ch = 0; ch < 3; ch++) c = fmax(c, fabs(S[order[k]].color[ch]));
    return c;
}

/* Renders the window [x0, x0+w) x [y0, y0+h) of the view.  image is [3][h][w].
   seq_hash (optional) receives an order-sensitive hash of each pixel's
   contributor sequence; ambiguity (optional, [2][h][w]) the bounds of
   pixel_walk for the colour and the final transmittance.  Returns the number
   of visible splats. */
ORC_API int64_t orc_render(const orc_gaussians *G, const orc_view *V, const orc_options *O, int x0, int y0,
                           int w, int h, int prefilter, double *image, double *T_final, int32_t *n_contrib,
                           uint8_t *flags, orc_splat *splats_out, uint64_t *seq_hash, double *ambiguity) {
    orc_splat *S = (orc_splat *)malloc(sizeof(orc_splat) * (G->n > 0 ? G->n : 1));
    int64_t *order;
    int64_t m = sorted_candidates(G, V, O, S, &order);
    const double cmax = max_color(S, order, m, V);
    int64_t nvis = 0;
    for (int64_t g = 0; g < G->n; g++) nvis += S[g].visible;
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            double C[3], T;
            uint8_t f;
            uint64_t hsh;
            double amb[2];
            int nc = pixel_walk(S, order, m, O, V, (double)(x0 + x), (double)(y0 + y), prefilter, C, &T, &f, NULL,
                                &hsh, amb, cmax);
            if (seq_hash) seq_hash[(int64_t)y * w + x] = hsh;
            if (ambiguity) {
                ambiguity[(int64_t)y * w + x] = amb[0];
                ambiguity[(int64_t)(h + y) * w + x] = amb[1];
            }
            for (int ch = 0; ch < 3; ch++) image[((int64_t)ch * h + y) * w + x] = C[ch];
            if (T_final) T_final[(int64_t)y * w + x] = T;
            if (n_contrib) n_contrib[(int64_t)y * w + x] = nc;
            if (flags) flags[(int64_t)y * w + x] = f;
        }
    if (splats_out) memcpy(splats_out, S, sizeof(orc_splat) * G->n);
    free(order);
    free(S);
    return nvis;
}

/* Eq. 6 with each splat's colour replaced by values[3 g + ch] and a zero
   background: the same walk, decisions and weights alpha_i T_i as the image,
   applied to other per-splat quantities (depth, flow).  out is [3][h][w]. */
ORC_API void orc_render_values(const orc_gaussians *G, const orc_view *V, const orc_options *O, int x0, int y0, int w,
                               int h, int prefilter, const double *values, double *out) {
    orc_splat *S = (orc_splat *)malloc(sizeof(orc_splat) * (G->n > 0 ? G->n : 1));
    int64_t *order;
    int64_t m = sorted_candidates(G, V, O, S, &order);
    for (int64_t g = 0; g < G->n; g++)
        for (int ch = 0; ch < 3; ch++) S[g].color[ch] = values[3 * g + ch];
    orc_view Vz = *V;
    for (int ch = 0; ch < 3; ch++) Vz.bg[ch] = 0.0;
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            double C[3], T;
            pixel_walk(S, order, m, O, &Vz, (double)(x0 + x), (double)(y0 + y), prefilter, C, &T, NULL, NULL, NULL,
                       NULL, 0.0);
            for (int ch = 0; ch < 3; ch++) out[((int64_t)ch * h + y) * w + x] = C[ch];
        }
    free(order);
    free(S);
}

/* ------------------------------------------------------------------ */
/* O9: hand-derived reverse mode                                        */
/* ------------------------------------------------------------------ */

/* grad2d layout per Gaussian (9 doubles):
   dL/du, dL/dv, dL/da, dL/db, dL/dc (conic), dL/dalpha_eff, dL/dcolor[3] */

/* Per-Gaussian chain rule from the 2D splat gradient back to the raw
   parameters (O6 -> O1).  g2d as above; accumulates into grads. */
ORC_API void orc_project_backward(const orc_gaussians *G, int64_t g, const orc_view *V, const orc_options *O,
                                  const double *g2d, orc_grads *grads) {
    const int64_t n = G->n;
    double mu[4], ls[4], ql[4], qr[4];
    for (int i = 0; i < 4; i++) {
        mu[i] = gparam(G->mu, i, g, n);
        ls[i] = gparam(G->log_s, i, g, n);
        ql[i] = gparam(G->ql, i, g, n);
        qr[i] = gparam(G->qr, i, g, n);
    }
    orc_splat S;
    if (!orc_project(G, g, V, O, &S)) return;

    /* ---- forward intermediates ---- */
    double s[4], qln[4], qrn[4], nl, nr, Lq[16], Rq[16], R[16], M[16], Mt[16], Sigma[16];
    for (int i = 0; i < 4; i++) s[i] = exp(ls[i]);
    normalize4(ql, qln, &nl);
    normalize4(qr, qrn, &nr);
    orc_quat_left(qln, Lq);
    orc_quat_right(qrn, Rq);
    matmul(Lq, Rq, R, 4, 4, 4);
    for (int i = 0; i < 4; i++)
        for (int k = 0; k < 4; k++) M[i * 4 + k] = R[i * 4 + k] * s[k];
    transpose(M, Mt, 4, 4);
    matmul(M, Mt, Sigma, 4, 4, 4);
    const double sig = Sigma[15];
    const double dt = V->t - mu[3];
    double b[3];
    for (int i = 0; i < 3; i++) b[i] = Sigma[i * 4 + 3];
    double W[9], Wt[9];
    for (int i = 0; i < 3; i++)
        for (int k = 0; k < 3; k++) W[i * 3 + k] = V->viewmat[i * 4 + k];
    transpose(W, Wt, 3, 3);
    const double X = S.xc[0], Y = S.xc[1], Z = S.xc[2];
    double J[6], T[6];
    int clx, cly;
    jacobian(V, O, S.xc, J, &clx, &cly);
    matmul(J, W, T, 2, 3, 3);

    /* ---- colour (Eq. 11) ---- */
    double dL_dmu3[3] = {0, 0, 0};
    double dL_ddt = 0.0; /* dt = t - mu_t */
    {
        const int nb = n_sh(G);
        double Cc[3], e[3], dir[3], nrm = 0.0;
        camera_center(V, Cc);
        for (int i = 0; i < 3; i++) { e[i] = S.mu3[i] - Cc[i]; nrm += e[i] * e[i]; }
        nrm = sqrt(nrm);
        for (int i = 0; i < 3; i++) dir[i] = e[i] / nrm;
        double Yb[64], dYb[192];
        orc_sh_basis(G->sh_degree, dir, Yb, dYb);
        double dL_ddir[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ch++) {
            /* colour = max(raw + 0.5, 0): gradient passes where raw + 0.5 > 0 */
            const double graw = (S.color_raw[ch] + 0.5 > 0.0) ? g2d[6 + ch] : 0.0;
            if (graw == 0.0) continue;
            for (int f = 0; f <= G->n_freq; f++) {
                const double w = 2.0 * M_PI * f / G->period;
                const double cf = cos(w * dt), sf = sin(w * dt);
                for (int j = 0; j < nb; j++) {
                    const int row = (f * nb + j) * 3 + ch;
                    const double k = gparam(G->shs, row, g, n);
                    grads->shs[(int64_t)row * n + g] += graw * cf * Yb[j];
                    dL_ddt += graw * (-w * sf) * k * Yb[j];
                    for (int i = 0; i < 3; i++) dL_ddir[i] += graw * cf * k * dYb[3 * j + i];
                }
            }
        }
        /* dir = e / |e|: project out the radial part */
        double dd = dL_ddir[0] * dir[0] + dL_ddir[1] * dir[1] + dL_ddir[2] * dir[2];
        for (int i = 0; i < 3; i++) dL_dmu3[i] += (dL_ddir[i] - dd * dir[i]) / nrm;
    }

    /* ---- conic -> 2D covariance (scalar form) ---- */
    const double S00 = S.cov2d[0], S01 = S.cov2d[1], S11 = S.cov2d[2];
    const double det = S00 * S11 - S01 * S01, det2 = det * det;
    const double ga = g2d[2], gb = g2d[3], gc = g2d[4];
    const double dS00 = ga * (-S11 * S11 / det2) + gb * (S01 * S11 / det2) + gc * (1.0 / det - S00 * S11 / det2);
    const double dS11 = ga * (1.0 / det - S11 * S00 / det2) + gb * (S01 * S00 / det2) + gc * (-S00 * S00 / det2);
    const double dS01 = ga * (2.0 * S11 * S01 / det2) + gb * (-1.0 / det - 2.0 * S01 * S01 / det2) +
                        gc * (2.0 * S00 * S01 / det2);
    /* full symmetric matrix gradient of Sigma_2d */
    const double G2[4] = {dS00, 0.5 * dS01, 0.5 * dS01, dS11};

    /* ---- Eq. 4: Sigma_2d = T Sigma3 T^T (+ delta I), T = J W ---- */
    double Tt[6], tmp32[6], GS3[9];
    transpose(T, Tt, 2, 3);
    matmul(Tt, G2, tmp32, 3, 2, 2);
    matmul(tmp32, T, GS3, 3, 2, 3); /* dL/dSigma3 = T^T G2 T */
    double G2T[6], dT[6], dJ[6];
    matmul(G2, T, G2T, 2, 2, 3);
    matmul(G2T, S.Sigma3, dT, 2, 3, 3);
    for (int i = 0; i < 6; i++) dT[i] *= 2.0; /* dL/dT = 2 G2 T Sigma3 */
    matmul(dT, Wt, dJ, 2, 3, 3);               /* dL/dJ = dL/dT W^T */

    /* ---- J and Eq. 3 (mean) w.r.t. camera coordinates ---- */
    double dxc[3] = {0, 0, 0};
    const double fx = V->fx, fy = V->fy;
    dxc[2] += dJ[0] * (-fx / (Z * Z)) + dJ[4] * (-fy / (Z * Z));
    {
        const double tx = clx ? -J[2] * Z / fx : X / Z; /* clamped or raw x/z */
        const double ty = cly ? -J[5] * Z / fy : Y / Z;
        /* J02 = -fx tx / Z, J12 = -fy ty / Z */
        dxc[2] += dJ[2] * (fx * tx / (Z * Z));
        dxc[2] += dJ[5] * (fy * ty / (Z * Z));
        if (!clx) {
            dxc[0] += dJ[2] * (-fx / Z) * (1.0 / Z);
            dxc[2] += dJ[2] * (-fx / Z) * (-X / (Z * Z));
        }
        if (!cly) {
            dxc[1] += dJ[5] * (-fy / Z) * (1.0 / Z);
            dxc[2] += dJ[5] * (-fy / Z) * (-Y / (Z * Z));
        }
    }
    const double gu = g2d[0], gv = g2d[1];
    dxc[0] += gu * fx / Z;
    dxc[2] += gu * (-fx * X / (Z * Z));
    dxc[1] += gv * fy / Z;
    dxc[2] += gv * (-fy * Y / (Z * Z));
    /* x_c = W mu3 + tau */
    for (int i = 0; i < 3; i++)
        for (int k = 0; k < 3; k++) dL_dmu3[i] += W[k * 3 + i] * dxc[k];

    /* ---- alpha_eff = alpha * p(t) ---- */
    const double galpha_eff = g2d[5];
    const double dL_dalpha = galpha_eff * S.p_t;
    const double dL_dp = galpha_eff * S.alpha;

    /* ---- Eq. 9 + Eq. 10 ---- */
    double dL_dA[9], dL_db[3], dL_dsig = 0.0;
    for (int i = 0; i < 9; i++) dL_dA[i] = GS3[i];
    for (int i = 0; i < 3; i++) {
        double Gb = 0.0;
        for (int k = 0; k < 3; k++) Gb += (GS3[i * 3 + k] + GS3[k * 3 + i]) * b[k];
        dL_db[i] = dL_dmu3[i] * dt / sig - Gb / sig;
    }
    {
        double mb = 0.0, bGb = 0.0;
        for (int i = 0; i < 3; i++) {
            mb += dL_dmu3[i] * b[i];
            for (int k = 0; k < 3; k++) bGb += b[i] * GS3[i * 3 + k] * b[k];
        }
        dL_dsig += -mb * dt / (sig * sig) + bGb / (sig * sig) + dL_dp * S.p_t * 0.5 * dt * dt / (sig * sig);
        dL_ddt += mb / sig + dL_dp * S.p_t * (-dt / sig);
    }
    /* dL/dmu */
    for (int i = 0; i < 3; i++) grads->mu[(int64_t)i * n + g] += dL_dmu3[i];
    grads->mu[(int64_t)3 * n + g] += -dL_ddt;

    /* full symmetric gradient of the 4x4 Sigma */
    double GS[16];
    for (int i = 0; i < 3; i++)
        for (int k = 0; k < 3; k++) GS[i * 4 + k] = dL_dA[i * 3 + k];
    for (int i = 0; i < 3; i++) { GS[i * 4 + 3] = 0.5 * dL_db[i]; GS[3 * 4 + i] = 0.5 * dL_db[i]; }
    GS[15] = dL_dsig;

    /* ---- Eq. 7: Sigma = M M^T, M = R diag(s) ---- */
    double GSs[16], dM[16];
    for (int i = 0; i < 4; i++)
        for (int k = 0; k < 4; k++) GSs[i * 4 + k] = GS[i * 4 + k] + GS[k * 4 + i];
    matmul(GSs, M, dM, 4, 4, 4);
    double dR[16];
    for (int i = 0; i < 4; i++)
        for (int k = 0; k < 4; k++) dR[i * 4 + k] = dM[i * 4 + k] * s[k];
    for (int k = 0; k < 4; k++) {
        double ds = 0.0;
        for (int i = 0; i < 4; i++) ds += dM[i * 4 + k] * R[i * 4 + k];
        grads->log_s[(int64_t)k * n + g] += ds * s[k];
    }
    /* ---- Eq. 8: R = L Rq ---- */
    double RqT[16], LT[16], dL_[16], dRq[16];
    transpose(Rq, RqT, 4, 4);
    transpose(Lq, LT, 4, 4);
    matmul(dR, RqT, dL_, 4, 4, 4);
    matmul(LT, dR, dRq, 4, 4, 4);
    /* entries of L(q) are +-q components: gradient = signed sums (Eq. 8 left matrix) */
    double gqln[4], gqrn[4];
    {
        const double *D = dL_;
        gqln[0] = D[0] + D[5] + D[10] + D[15];
        gqln[1] = -D[1] + D[4] - D[11] + D[14];
        gqln[2] = -D[2] + D[7] + D[8] - D[13];
        gqln[3] = -D[3] - D[6] + D[9] + D[12];
        const double *E = dRq;
        gqrn[0] = E[0] + E[5] + E[10] + E[15];
        gqrn[1] = -E[1] + E[4] + E[11] - E[14];
        gqrn[2] = -E[2] - E[7] + E[8] + E[13];
        gqrn[3] = -E[3] + E[6] - E[9] + E[12];
    }
    /* q_hat = q / |q| */
    double dl = 0.0, dr = 0.0;
    for (int i = 0; i < 4; i++) { dl += gqln[i] * qln[i]; dr += gqrn[i] * qrn[i]; }
    for (int i = 0; i < 4; i++) {
        grads->ql[(int64_t)i * n + g] += (gqln[i] - dl * qln[i]) / nl;
        grads->qr[(int64_t)i * n + g] += (gqrn[i] - dr * qrn[i]) / nr;
    }
    /* alpha = sigmoid(logit) */
    grads->logit[g] += dL_dalpha * S.alpha * (1.0 - S.alpha);
}

/* Backward of orc_render over the window; dL_dimage is [3][h][w].
   grad2d (optional, [n][9]) receives the per-splat 2D gradients (+=). */
ORC_API void orc_backward(const orc_gaussians *G, const orc_view *V, const orc_options *O, int x0, int y0,
                          int w, int h, int prefilter, const double *dL_dimage, orc_grads *grads,
                          double *grad2d) {
    const int64_t n = G->n;
    orc_splat *S = (orc_splat *)malloc(sizeof(orc_splat) * (n > 0 ? n : 1));
    int64_t *order;
    int64_t m = sorted_candidates(G, V, O, S, &order);
    double *g2 = (double *)calloc((size_t)(n > 0 ? n : 1) * 9, sizeof(double));
    contrib *list = (contrib *)malloc(sizeof(contrib) * (m > 0 ? m : 1));
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            double C[3], T;
            int nc = pixel_walk(S, order, m, O, V, (double)(x0 + x), (double)(y0 + y), prefilter, C, &T, NULL, list,
                                NULL, NULL, 0.0);
            double dC[3];
            for (int ch = 0; ch < 3; ch++) dC[ch] = dL_dimage[((int64_t)ch * h + y) * w + x];
            /* acc = sum_{j>i} c_j alpha_j T_j + T_final bg, built back to front */
            double acc[3];
            for (int ch = 0; ch < 3; ch++) acc[ch] = T * V->bg[ch];
            for (int i = nc - 1; i >= 0; i--) {
                const contrib *c = &list[i];
                const orc_splat *s = &S[c->g];
                double *gg = &g2[c->g * 9];
                double dalpha = 0.0;
                for (int ch = 0; ch < 3; ch++) {
                    gg[6 + ch] += dC[ch] * c->alpha * c->T;
                    dalpha += dC[ch] * (s->color[ch] * c->T - acc[ch] / (1.0 - c->alpha));
                    acc[ch] += s->color[ch] * c->alpha * c->T;
                }
                if (c->clamped) continue; /* alpha = alpha_max: no dependence */
                gg[5] += dalpha * c->Gexp;
                const double dpow = dalpha * c->araw;
                const double dx = c->dx, dy = c->dy;
                gg[2] += dpow * (-0.5 * dx * dx);
                gg[4] += dpow * (-0.5 * dy * dy);
                gg[3] += dpow * (-dx * dy);
                gg[0] += dpow * (s->conic[0] * dx + s->conic[1] * dy);
                gg[1] += dpow * (s->conic[2] * dy + s->conic[1] * dx);
            }
        }
    for (int64_t g = 0; g < n; g++) {
        if (!S[g].visible) continue;
        orc_project_backward(G, g, V, O, &g2[g * 9], grads);
        if (grad2d)
            for (int k = 0; k < 9; k++) grad2d[g * 9 + k] += g2[g * 9 + k];
    }
    free(list);
    free(g2);
    free(order);
    free(S);
}

ORC_API int orc_splat_size(void) { return (int)sizeof(orc_splat); }
