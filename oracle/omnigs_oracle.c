/*
 * omnigs_oracle.c -- plain, slow FP64 CPU oracle of equirectangular Gaussian splatting (OmniGS, arXiv 2404.03202).
 *
 * TEST INFRASTRUCTURE. This library exists to check the CUDA path. Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it; the product path never does. It shares no code, header, table or
 * helper with the CUDA sources.
 *
 * Every function follows one passage of the paper, in the paper's order and notation:
 *   t = W m + t_cw                                   (Sec. 3.2, Eq. 1)
 *   lon = atan2(t_x, t_z), lat = asin(t_y / t_r)      (Sec. 3.2, Eq. 3)
 *   s = (lon / pi, 2 lat / pi)                        (Sec. 3.2, Eq. 4)
 *   p = ((s_x + 1) W / 2, (s_y + 1) H / 2)            (Sec. 3.2, Eq. 5)
 *   C = sum_i c_i a_i prod_{j<i} (1 - a_j), sorted by t_r           (Sec. 3.3, Eq. 6)
 *   a_i = o_i G_i(dp),  G = exp(-1/2 dp^T Sigma~^-1 dp)             (Sec. 3.3, Eqs. 7-8)
 *   Sigma~ = J W Sigma W^T J^T, 2x2 block kept                       (Sec. 3.3, Eqs. 9-16)
 *   tile-based procedure, stop at accumulated alpha 0.9999          (Sec. 3.3, last paragraph)
 *   gradients by the chain rule through J, p, s and t               (Sec. 3.4, Eqs. 18-20)
 *
 * Readings of points the paper leaves open (each is a convention of the 3DGS renderer the paper builds on):
 *   - Eq. 3 prints "arctan2(t_x / t_z)"; it is read as the two-argument atan2(t_x, t_z), the only reading that
 *     agrees with dp_x/dt_x = +W/(2 pi) t_z/(t_x^2 + t_z^2) of Eq. 11. lon = +pi is mapped to -pi (lon in [-pi, pi)).
 *   - Eq. 10 prints dp_y/dt_y twice in its second row; the third entry is dp_y/dt_z (Eq. 16).
 *   - near cull t_r <= near_r; low-pass dilation Sigma~ += 0.3 I; cull if det(Sigma~) <= 0.
 *   - radius of influence r = ceil(3 sqrt(lambda_max)), lambda_max = mid + sqrt(max(0.1, mid^2 - det)).
 *   - instances come from the box of half-extents (rx, ry) around pixel floor(p): the square of half-side r,
 *     narrowed per axis to the box of the region where alpha >= 1/255: with q = 2 ln(255 o), that region is the
 *     ellipse dp^T Sigma~^-1 dp <= q, whose half-extents are sqrt(q Sigma~_00) and sqrt(q Sigma~_11);
 *     rx = min(r, ceil(sqrt(q Sigma~_00) (1 + 1e-4) + 1e-3)), ry likewise (the small widening absorbs FP32
 *     rounding on the GPU). A Gaussian with 255 o < 1 has no instance. Outside that box alpha < 1/255 at every
 *     pixel, so the narrowing leaves every image unchanged; it only drops instances that contribute nothing.
 *     rx and ry are held at 65535 (images are at most 65536 px a side, so for the equirectangular camera a held box
 *     still spans every column and row it reaches).
 *   - one instance per (Gaussian, tile) pair for every tile the box touches: these are the lists this oracle builds.
 *     An implementation may leave out pairs whose tile has no pixel centre with alpha >= 1/255 (they change no
 *     pixel); the test-suite checks such lists against these (tests/tile_check.py).
 *   - quaternion stored (w, x, y, z), normalised before use; Sigma = R diag(s)^2 R^T.
 *   - colour c = max(sum_k Y_k(d) sh_k + 0.5, 0) with d the unit vector from the camera centre to m and Y_k the real
 *     orthonormal spherical harmonics up to degree 3 (no Condon-Shortley phase).
 *   - pixel (x, y) is sampled at its centre (x + 0.5, y + 0.5); dp_x is taken as the minimal image in [-W/2, W/2)
 *     (the longitude seam); tile columns wrap modulo the tile count; rows are clamped (no wrap over the poles).
 *   - alpha = min(0.99, o G); skip if G's exponent > 0 or alpha < 1/255; stop before a Gaussian whose
 *     T (1 - alpha) < 1e-4; background bg added with the final T.
 *   - the gradient is the exact derivative of the above (zero where alpha is clamped at 0.99 or a colour at 0).
 *   - pole guard: rho = sqrt(t_x^2 + t_z^2) is replaced by max(rho, 1e-6 t_r) inside J.
 *
 * Pinhole camera (Eq. 2, the perspective model of 3DGS the paper contrasts with; selected by orc_set_camera):
 *   p = (f_x t_x / t_z + c_x, f_y t_y / t_z + c_y); the depth that orders Gaussians is t_z; near cull t_z <= near_r;
 *   J = [[f_x / t_z, 0, -f_x u / t_z], [0, f_y / t_z, -f_y w / t_z]] with u = clamp(t_x / t_z, +-1.3 W / (2 f_x))
 *   and w = clamp(t_y / t_z, +-1.3 H / (2 f_y)) (the 3DGS guard that keeps J bounded off screen), while dp/dt, the
 *   derivative of p itself, is unclamped; tile columns are clipped like rows and dx is not wrapped; a Gaussian whose
 *   instance box [floor(p_x) - r_x, floor(p_x) + r_x] x [floor(p_y) - r_y, floor(p_y) + r_y] misses the image
 *   [0, W) x [0, H) is culled (the frustum cull of 3DGS: such a Gaussian has no tile, hence no instance, either way).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define ORC_DILATION 0.3
#define ORC_ALPHA_MAX 0.99
#define ORC_ALPHA_MIN (1.0 / 255.0)
#define ORC_T_STOP 1e-4
#define ORC_POLE_GUARD 1e-6
/* unit roundoff of single precision, 2^-24: the near-threshold flags of orc_blend_fwd widen by the rounding error a
 * single-precision evaluation of the exponent can make (a few roundoffs of the magnitude of its terms) */
#define ORC_F32_ROUNDOFF 5.9604644775390625e-8

/* per-(view, Gaussian) record written by orc_preprocess. R_RADIUS is the square's r; R_RX, R_RY the half-extents
 * of the box the instances come from; R_RMARGIN the smallest distance of the three ceil() arguments to an integer. */
enum {
    R_PX = 0, R_PY, R_DEPTH, R_C0, R_C1, R_C2, R_OPAC, R_RED, R_GREEN, R_BLUE, R_RADIUS,
    R_COV00, R_COV01, R_COV11, R_RMARGIN, R_FLAGS, R_RX, R_RY, R_Q, R_LEN
};
/* per-(view, Gaussian) screen-space gradient, written by orc_blend_bwd and read by orc_preprocess_bwd */
enum { G_PX = 0, G_PY, G_C0, G_C1, G_C2, G_OPAC, G_RED, G_GREEN, G_BLUE, G_LEN };

int orc_record_len(void) { return R_LEN; }
int orc_grad_len(void) { return G_LEN; }

/* ------------------------------------------------------------------ camera model */
typedef struct { int model; double fx, fy, cx, cy; } orc_cam;  /* model 0: equirectangular, 1: pinhole */
static orc_cam g_cam = {0, 0.0, 0.0, 0.0, 0.0};

void orc_set_camera(int model, double fx, double fy, double cx, double cy)
{
    g_cam.model = model; g_cam.fx = fx; g_cam.fy = fy; g_cam.cx = cx; g_cam.cy = cy;
}

/* ------------------------------------------------------------------ Eqs. 3-5: t -> (lon, lat) -> s -> p */
void orc_project(const double *t, int W, int H, double *lonlat, double *s, double *p)
{
    double tr = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    double lon = atan2(t[0], t[2]);
    if (lon >= ORC_PI) lon = -ORC_PI;
    double q = t[1] / tr;
    if (q > 1.0) q = 1.0;
    if (q < -1.0) q = -1.0;
    double lat = asin(q);
    lonlat[0] = lon;
    lonlat[1] = lat;
    s[0] = lon / ORC_PI;
    s[1] = 2.0 * lat / ORC_PI;
    p[0] = (s[0] + 1.0) * W / 2.0;
    p[1] = (s[1] + 1.0) * H / 2.0;
}

/* ------------------------------------------------------------------ Eqs. 10-16: J = dp/dt (2 x 3, row-major) */
static double guarded_rho(const double *t, double tr)
{
    double rho = sqrt(t[0] * t[0] + t[2] * t[2]);
    double g = ORC_POLE_GUARD * tr;
    return rho > g ? rho : g;
}

void orc_jacobian(const double *t, int W, int H, double *J)
{
    double a = W / (2.0 * ORC_PI), b = H / ORC_PI;
    double tr = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    double rho = guarded_rho(t, tr);
    double tr2 = tr * tr;
    J[0] = a * t[2] / (rho * rho);                 /* Eq. 11 */
    J[1] = 0.0;                                    /* Eq. 12 */
    J[2] = -a * t[0] / (rho * rho);                /* Eq. 13 */
    J[3] = -b * t[0] * t[1] / (tr2 * rho);         /* Eq. 14 */
    J[4] = b * rho / tr2;                          /* Eq. 15 */
    J[5] = -b * t[2] * t[1] / (tr2 * rho);         /* Eq. 16 */
}

/* dJ/dt: dJ[r][c][k] = d J_rc / d t_k, the derivative of orc_jacobian (the supplement's derivation is not
 * available, so it is derived here by the quotient rule). */
static void jacobian_grad(const double *t, int W, int H, double dJ[2][3][3])
{
    double a = W / (2.0 * ORC_PI), b = H / ORC_PI;
    double tr = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    double rho_true = sqrt(t[0] * t[0] + t[2] * t[2]);
    double rho = guarded_rho(t, tr);
    double drho[3], dtr[3];
    if (rho_true >= ORC_POLE_GUARD * tr) {
        drho[0] = t[0] / rho; drho[1] = 0.0; drho[2] = t[2] / rho;
    } else {
        drho[0] = ORC_POLE_GUARD * t[0] / tr; drho[1] = ORC_POLE_GUARD * t[1] / tr; drho[2] = ORC_POLE_GUARD * t[2] / tr;
    }
    for (int k = 0; k < 3; k++) dtr[k] = t[k] / tr;
    double tr2 = tr * tr, tr3 = tr2 * tr, rho2 = rho * rho, rho3 = rho2 * rho;
    for (int k = 0; k < 3; k++) {
        double ex = (k == 0), ey = (k == 1), ez = (k == 2);
        dJ[0][0][k] = a * (ez / rho2 - 2.0 * t[2] * drho[k] / rho3);
        dJ[0][1][k] = 0.0;
        dJ[0][2][k] = -a * (ex / rho2 - 2.0 * t[0] * drho[k] / rho3);
        dJ[1][0][k] = -b * ((t[1] * ex + t[0] * ey) / (tr2 * rho) - 2.0 * t[0] * t[1] * dtr[k] / (tr3 * rho)
                            - t[0] * t[1] * drho[k] / (tr2 * rho2));
        dJ[1][1][k] = b * (drho[k] / tr2 - 2.0 * rho * dtr[k] / tr3);
        dJ[1][2][k] = -b * ((t[1] * ez + t[2] * ey) / (tr2 * rho) - 2.0 * t[2] * t[1] * dtr[k] / (tr3 * rho)
                            - t[2] * t[1] * drho[k] / (tr2 * rho2));
    }
}

/* dJ/dt of the pinhole Jacobian (Eq. 2) with its clamped ratios: a clamped ratio is a constant. */
static void pinhole_jacobian_grad(const double *t, int W, int H, double dJ[2][3][3])
{
    double tz = t[2], fx = g_cam.fx, fy = g_cam.fy;
    double limx = 1.3 * W / (2.0 * fx), limy = 1.3 * H / (2.0 * fy);
    double u = t[0] / tz, w = t[1] / tz;
    int cu = u < -limx || u > limx, cw = w < -limy || w > limy;
    double uc = u < -limx ? -limx : (u > limx ? limx : u), wc = w < -limy ? -limy : (w > limy ? limy : w);
    memset(dJ, 0, sizeof(double) * 18);
    dJ[0][0][2] = -fx / (tz * tz);
    dJ[1][1][2] = -fy / (tz * tz);
    /* J02 = -fx u / tz: unclamped u = tx / tz gives -fx tx / tz^2 */
    if (cu) dJ[0][2][2] = fx * uc / (tz * tz);
    else { dJ[0][2][0] = -fx / (tz * tz); dJ[0][2][2] = 2.0 * fx * t[0] / (tz * tz * tz); }
    if (cw) dJ[1][2][2] = fy * wc / (tz * tz);
    else { dJ[1][2][1] = -fy / (tz * tz); dJ[1][2][2] = 2.0 * fy * t[1] / (tz * tz * tz); }
}

/* ------------------------------------------------------------------ Sec. 3.1: colour from SH (real basis) */
/* Real orthonormal spherical harmonics of degree <= 3 at unit direction d = (x, y, z); constants from
 * Y_lm normalisation sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times the real-form factors. */
void orc_sh_basis(int degree, const double *d, double *Y, double *dY /* [16][3] or NULL */)
{
    double x = d[0], y = d[1], z = d[2];
    double k0 = 0.5 * sqrt(1.0 / ORC_PI);
    double k1 = sqrt(3.0 / (4.0 * ORC_PI));
    double k2a = 0.5 * sqrt(15.0 / ORC_PI), k2b = 0.25 * sqrt(5.0 / ORC_PI), k2c = 0.25 * sqrt(15.0 / ORC_PI);
    double k3a = 0.25 * sqrt(35.0 / (2.0 * ORC_PI)), k3b = 0.5 * sqrt(105.0 / ORC_PI);
    double k3c = 0.25 * sqrt(21.0 / (2.0 * ORC_PI)), k3d = 0.25 * sqrt(7.0 / ORC_PI), k3e = 0.25 * sqrt(105.0 / ORC_PI);
    double g[16][3];
    memset(g, 0, sizeof(g));
    for (int i = 0; i < 16; i++) Y[i] = 0.0;
    Y[0] = k0;
    if (degree >= 1) {
        Y[1] = k1 * y; g[1][1] = k1;
        Y[2] = k1 * z; g[2][2] = k1;
        Y[3] = k1 * x; g[3][0] = k1;
    }
    if (degree >= 2) {
        Y[4] = k2a * x * y;               g[4][0] = k2a * y; g[4][1] = k2a * x;
        Y[5] = k2a * y * z;               g[5][1] = k2a * z; g[5][2] = k2a * y;
        Y[6] = k2b * (3.0 * z * z - 1.0); g[6][2] = 6.0 * k2b * z;
        Y[7] = k2a * x * z;               g[7][0] = k2a * z; g[7][2] = k2a * x;
        Y[8] = k2c * (x * x - y * y);     g[8][0] = 2.0 * k2c * x; g[8][1] = -2.0 * k2c * y;
    }
    if (degree >= 3) {
        Y[9] = k3a * y * (3.0 * x * x - y * y);
        g[9][0] = 6.0 * k3a * x * y; g[9][1] = k3a * (3.0 * x * x - 3.0 * y * y);
        Y[10] = k3b * x * y * z;
        g[10][0] = k3b * y * z; g[10][1] = k3b * x * z; g[10][2] = k3b * x * y;
        Y[11] = k3c * y * (5.0 * z * z - 1.0);
        g[11][1] = k3c * (5.0 * z * z - 1.0); g[11][2] = 10.0 * k3c * y * z;
        Y[12] = k3d * z * (5.0 * z * z - 3.0);
        g[12][2] = k3d * (15.0 * z * z - 3.0);
        Y[13] = k3c * x * (5.0 * z * z - 1.0);
        g[13][0] = k3c * (5.0 * z * z - 1.0); g[13][2] = 10.0 * k3c * x * z;
        Y[14] = k3e * z * (x * x - y * y);
        g[14][0] = 2.0 * k3e * x * z; g[14][1] = -2.0 * k3e * y * z; g[14][2] = k3e * (x * x - y * y);
        Y[15] = k3a * x * (x * x - 3.0 * y * y);
        g[15][0] = k3a * (3.0 * x * x - 3.0 * y * y); g[15][1] = -6.0 * k3a * x * y;
    }
    if (dY) memcpy(dY, g, sizeof(g));
}

/* ------------------------------------------------------------------ Sec. 3.3: Sigma from (q, S) */
void orc_quat_to_rot(const double *q_in, double *R)
{
    double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
    R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z);       R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);       R[7] = 2.0 * (y * z + w * x);       R[8] = 1.0 - 2.0 * (x * x + y * y);
}

/* dR_ij / d(w, x, y, z) of the unit quaternion */
static void rot_grad(const double *qn, double dR[9][4])
{
    double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    double t[9][4] = {
        {0, 0, -4 * y, -4 * z},
        {-2 * z, 2 * y, 2 * x, -2 * w},
        {2 * y, 2 * z, 2 * w, 2 * x},
        {2 * z, 2 * y, 2 * x, 2 * w},
        {0, -4 * x, 0, -4 * z},
        {-2 * x, -2 * w, 2 * z, 2 * y},
        {-2 * y, 2 * z, -2 * w, 2 * x},
        {2 * x, 2 * w, 2 * z, 2 * y},
        {0, -4 * x, -4 * y, 0},
    };
    memcpy(dR, t, sizeof(t));
}

/* 3D covariance Sigma = R diag(s)^2 R^T */
static void covariance3d(const double *q, const double *s, double *Sig, double *R)
{
    orc_quat_to_rot(q, R);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += R[i * 3 + k] * s[k] * s[k] * R[j * 3 + k];
            Sig[i * 3 + j] = acc;
        }
}

/* ------------------------------------------------------------------ per-(view, Gaussian) forward quantities */
typedef struct {
    int culled;
    double t[3], tr, p[2], J[6], Jp[6], Wr[9], M[6], Sig[9], R[9], cov[3], det, conic[3], radius, rx, ry, rmargin, q;
    double dir[3], dist, Y[16], rgb_raw[3], rgb[3];
} orc_fwd;

static void load_view(const float *viewmat, double *Wr, double *tcw, double *campos)
{
    for (int i = 0; i < 3; i++) {
        for (int j = 0; j < 3; j++) Wr[i * 3 + j] = viewmat[i * 4 + j];
        tcw[i] = viewmat[i * 4 + 3];
    }
    /* camera centre in world coordinates: c = -W^T t_cw */
    for (int j = 0; j < 3; j++) campos[j] = -(Wr[0 * 3 + j] * tcw[0] + Wr[1 * 3 + j] * tcw[1] + Wr[2 * 3 + j] * tcw[2]);
}

static double int_gap(double z) { return fabs(z - floor(z + 0.5)); }

static void forward_one(int W, int H, int sh_degree, double near_r, const float *m_f, const float *s_f,
                        const float *q_f, const float *sh_f, double opacity, const double *Wr, const double *tcw,
                        const double *campos, orc_fwd *f)
{
    int K = (sh_degree + 1) * (sh_degree + 1);
    double m[3] = {m_f[0], m_f[1], m_f[2]}, s[3] = {s_f[0], s_f[1], s_f[2]};
    double q[4] = {q_f[0], q_f[1], q_f[2], q_f[3]};
    memset(f, 0, sizeof(*f));
    memcpy(f->Wr, Wr, sizeof(double) * 9);
    /* Eq. 1 */
    for (int i = 0; i < 3; i++) f->t[i] = Wr[i * 3 + 0] * m[0] + Wr[i * 3 + 1] * m[1] + Wr[i * 3 + 2] * m[2] + tcw[i];
    if (g_cam.model == 1) {
        /* Eq. 2 and its Jacobian; the depth that orders Gaussians is t_z */
        double tz = f->t[2];
        f->tr = tz;
        if (tz <= near_r) { f->culled = 1; return; }
        f->p[0] = g_cam.fx * f->t[0] / tz + g_cam.cx;
        f->p[1] = g_cam.fy * f->t[1] / tz + g_cam.cy;
        double limx = 1.3 * W / (2.0 * g_cam.fx), limy = 1.3 * H / (2.0 * g_cam.fy);
        double u = f->t[0] / tz, w = f->t[1] / tz;
        u = u < -limx ? -limx : (u > limx ? limx : u);
        w = w < -limy ? -limy : (w > limy ? limy : w);
        f->J[0] = g_cam.fx / tz; f->J[1] = 0.0; f->J[2] = -g_cam.fx * u / tz;
        f->J[3] = 0.0; f->J[4] = g_cam.fy / tz; f->J[5] = -g_cam.fy * w / tz;
        f->Jp[0] = g_cam.fx / tz; f->Jp[1] = 0.0; f->Jp[2] = -g_cam.fx * f->t[0] / (tz * tz);
        f->Jp[3] = 0.0; f->Jp[4] = g_cam.fy / tz; f->Jp[5] = -g_cam.fy * f->t[1] / (tz * tz);
    } else {
        f->tr = sqrt(f->t[0] * f->t[0] + f->t[1] * f->t[1] + f->t[2] * f->t[2]);
        if (f->tr <= near_r) { f->culled = 1; return; }
        /* Eqs. 3-5 and 10-16 */
        double lonlat[2], sv[2];
        orc_project(f->t, W, H, lonlat, sv, f->p);
        orc_jacobian(f->t, W, H, f->J);
        memcpy(f->Jp, f->J, sizeof(f->J));
    }
    /* Eq. 9: Sigma~ = (J W) Sigma (J W)^T, 2x2 block, plus the low-pass dilation */
    covariance3d(q, s, f->Sig, f->R);
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++)
            f->M[r * 3 + c] = f->J[r * 3 + 0] * Wr[0 * 3 + c] + f->J[r * 3 + 1] * Wr[1 * 3 + c] + f->J[r * 3 + 2] * Wr[2 * 3 + c];
    double cv[2][2];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 2; c++) {
            double acc = 0.0;
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) acc += f->M[r * 3 + i] * f->Sig[i * 3 + j] * f->M[c * 3 + j];
            cv[r][c] = acc;
        }
    f->cov[0] = cv[0][0] + ORC_DILATION;
    f->cov[1] = cv[0][1];
    f->cov[2] = cv[1][1] + ORC_DILATION;
    f->det = f->cov[0] * f->cov[2] - f->cov[1] * f->cov[1];
    if (f->det <= 0.0) { f->culled = 1; return; }
    f->conic[0] = f->cov[2] / f->det;
    f->conic[1] = -f->cov[1] / f->det;
    f->conic[2] = f->cov[0] / f->det;
    double mid = 0.5 * (f->cov[0] + f->cov[2]);
    double disc = mid * mid - f->det;
    double lam = mid + sqrt(disc > 0.1 ? disc : 0.1);
    double rr = 3.0 * sqrt(lam);
    f->radius = ceil(rr);
    /* the box of the alpha >= 1/255 ellipse, widened slightly; no instance at all when 255 o < 1 */
    double qa = 2.0 * log(255.0 * opacity);
    if (255.0 * opacity < 1.0) { f->culled = 1; return; }
    if (qa < 0.0) qa = 0.0;
    double hx = sqrt(qa * f->cov[0]) * (1.0 + 1e-4) + 1e-3, hy = sqrt(qa * f->cov[2]) * (1.0 + 1e-4) + 1e-3;
    f->rx = ceil(hx) < f->radius ? ceil(hx) : f->radius;
    f->ry = ceil(hy) < f->radius ? ceil(hy) : f->radius;
    if (f->rx > 65535.0) f->rx = 65535.0;
    if (f->ry > 65535.0) f->ry = 65535.0;
    if (g_cam.model == 1) { /* pinhole: a box that misses the image has no tile */
        double ix = floor(f->p[0]), iy = floor(f->p[1]);
        if (ix + f->rx < 0.0 || ix - f->rx >= (double)W || iy + f->ry < 0.0 || iy - f->ry >= (double)H) {
            f->culled = 1;
            return;
        }
    }
    f->q = qa;
    f->rmargin = fmin(int_gap(rr), fmin(int_gap(hx), int_gap(hy)));
    /* Sec. 3.1: colour from m and the SH coefficients */
    double v[3] = {m[0] - campos[0], m[1] - campos[1], m[2] - campos[2]};
    f->dist = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int i = 0; i < 3; i++) f->dir[i] = v[i] / f->dist;
    orc_sh_basis(sh_degree, f->dir, f->Y, NULL);
    for (int ch = 0; ch < 3; ch++) {
        double acc = 0.0;
        for (int k = 0; k < K; k++) acc += f->Y[k] * sh_f[k * 3 + ch];
        f->rgb_raw[ch] = acc + 0.5;
        f->rgb[ch] = f->rgb_raw[ch] > 0.0 ? f->rgb_raw[ch] : 0.0;
    }
}

/* Projection of every (view, Gaussian) pair. rec: [V * n][R_LEN] doubles, index v * n + g. */
void orc_preprocess(int64_t n, int V, int W, int H, int sh_degree, double near_r,
                    const float *means, const float *scales, const float *quats, const float *opacity,
                    const float *sh, const float *viewmats, double *rec)
{
    int K = (sh_degree + 1) * (sh_degree + 1);
    for (int v = 0; v < V; v++) {
        double Wr[9], tcw[3], campos[3];
        load_view(viewmats + 16 * v, Wr, tcw, campos);
        for (int64_t g = 0; g < n; g++) {
            orc_fwd f;
            forward_one(W, H, sh_degree, near_r, means + 3 * g, scales + 3 * g, quats + 4 * g, sh + 3 * K * g,
                        opacity[g], Wr, tcw, campos, &f);
            double *o = rec + (int64_t)R_LEN * (v * n + g);
            memset(o, 0, sizeof(double) * R_LEN);
            o[R_DEPTH] = f.tr;
            if (f.culled) { o[R_FLAGS] = 1.0; continue; }
            o[R_PX] = f.p[0]; o[R_PY] = f.p[1];
            o[R_C0] = f.conic[0]; o[R_C1] = f.conic[1]; o[R_C2] = f.conic[2];
            o[R_OPAC] = opacity[g];
            o[R_RED] = f.rgb[0]; o[R_GREEN] = f.rgb[1]; o[R_BLUE] = f.rgb[2];
            o[R_RADIUS] = f.radius;
            o[R_COV00] = f.cov[0]; o[R_COV01] = f.cov[1]; o[R_COV11] = f.cov[2];
            o[R_RMARGIN] = f.rmargin;
            o[R_RX] = f.rx; o[R_RY] = f.ry; o[R_Q] = f.q;
        }
    }
}

/* ------------------------------------------------------------------ Sec. 3.3: tiles, instances, sort by t_r */
static int64_t floordiv(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q--;
    return q;
}

/* Tile rectangle covered by the box of half-extents (rx, ry) around pixel floor(p). Columns start at x0 and run
 * nx columns modulo the tile-column count (the longitude seam); rows y0..y0+ny-1 are clamped to the image. */
void orc_rect(double px, double py, int rx, int ry, int W, int H, int T, int64_t *out /* x0, nx, y0, ny */)
{
    int64_t TX = W / T, TY = H / T;
    int64_t ix = (int64_t)floor(px), iy = (int64_t)floor(py);
    int64_t x0 = floordiv(ix - rx, T), x1 = floordiv(ix + rx, T);
    if (g_cam.model == 1) { /* pinhole: columns clipped like rows */
        if (x0 < 0) x0 = 0;
        if (x1 > TX - 1) x1 = TX - 1;
    }
    int64_t nx = x1 - x0 + 1;
    if (nx < 0) nx = 0;
    if (nx >= TX) { x0 = 0; nx = TX; }
    int64_t y0 = floordiv(iy - ry, T), y1 = floordiv(iy + ry, T);
    if (y0 < 0) y0 = 0;
    if (y1 > TY - 1) y1 = TY - 1;
    out[0] = x0; out[1] = nx; out[2] = y0; out[3] = y1 - y0 + 1;
    if (out[3] < 0) out[3] = 0;
}

typedef struct { int64_t tile; double depth; int64_t vg; } orc_inst;

static int inst_cmp(const void *a, const void *b)
{
    const orc_inst *x = (const orc_inst *)a, *y = (const orc_inst *)b;
    if (x->tile != y->tile) return x->tile < y->tile ? -1 : 1;
    if (x->depth != y->depth) return x->depth < y->depth ? -1 : 1;
    if (x->vg != y->vg) return x->vg < y->vg ? -1 : 1;
    return 0;
}

/* Instances of one splat: every tile of its box (Sec. 3.3, one instance per influence), row by row. */
static int64_t splat_instances(double px, double py, int rx, int ry, int W, int H, int T,
                               int64_t *tiles_out /* NULL: count only */)
{
    int64_t TX = W / T, r[4], k = 0;
    orc_rect(px, py, rx, ry, W, H, T, r);
    for (int64_t ty = r[2]; ty < r[2] + r[3]; ty++)
        for (int64_t c = r[0]; c < r[0] + r[1]; c++) {
            if (tiles_out) tiles_out[k] = ty * TX + ((c % TX) + TX) % TX;
            k++;
        }
    return k;
}

int64_t orc_count_instances(int V, int64_t n, int W, int H, int T, const double *px, const double *py,
                            const int32_t *rx, const int32_t *ry)
{
    int64_t total = 0;
    for (int64_t i = 0; i < (int64_t)V * n; i++) {
        if (rx[i] <= 0) continue;
        total += splat_instances(px[i], py[i], rx[i], ry[i], W, H, T, NULL);
    }
    return total;
}

/* One instance per (Gaussian, tile of its box); order by (view, tile), then t_r, then Gaussian index (the order a stable
 * sort by (tile, t_r) gives when instances are generated Gaussian by Gaussian). ranges: [V*TX*TY][2].
 * tile_mask (optional, [V*TX*TY]): when given, only instances of tiles whose mask byte is non-zero are listed
 * (the lists of those tiles are the same as without a mask). Returns the number of listed instances; with
 * list_vg == NULL it only counts them. */
int64_t orc_bin_sort(int V, int64_t n, int W, int H, int T, const double *px, const double *py,
                     const int32_t *rx, const int32_t *ry, const double *depth, int64_t *ranges, int64_t *list_vg,
                     const uint8_t *tile_mask)
{
    int64_t TX = W / T, TY = H / T, tiles = TX * TY;
    int64_t *buf = (int64_t *)malloc(sizeof(int64_t) * (size_t)(tiles > 0 ? tiles : 1));
    int64_t total = 0;
    for (int v = 0; v < V; v++)
        for (int64_t g = 0; g < n; g++) {
            int64_t i = v * n + g;
            if (rx[i] <= 0) continue;
            int64_t m = splat_instances(px[i], py[i], rx[i], ry[i], W, H, T, buf);
            for (int64_t k = 0; k < m; k++) total += !tile_mask || tile_mask[v * tiles + buf[k]];
        }
    if (!list_vg) { free(buf); return total; } /* count only */
    orc_inst *inst = (orc_inst *)malloc(sizeof(orc_inst) * (total > 0 ? total : 1));
    int64_t k = 0;
    for (int v = 0; v < V; v++)
        for (int64_t g = 0; g < n; g++) {
            int64_t i = v * n + g;
            if (rx[i] <= 0) continue;
            int64_t m = splat_instances(px[i], py[i], rx[i], ry[i], W, H, T, buf);
            for (int64_t e = 0; e < m; e++) {
                int64_t t = v * tiles + buf[e];
                if (tile_mask && !tile_mask[t]) continue;
                inst[k].tile = t;
                inst[k].depth = depth[i];
                inst[k].vg = i;
                k++;
            }
        }
    qsort(inst, (size_t)total, sizeof(orc_inst), inst_cmp);
    for (int64_t t = 0; t < (int64_t)V * tiles; t++) { ranges[2 * t] = 0; ranges[2 * t + 1] = 0; }
    for (int64_t j = 0; j < total; j++) {
        list_vg[j] = inst[j].vg;
        int64_t t = inst[j].tile;
        if (j == 0 || inst[j - 1].tile != t) ranges[2 * t] = j;
        if (j == total - 1 || inst[j + 1].tile != t) ranges[2 * t + 1] = j + 1;
    }
    free(inst);
    free(buf);
    return total;
}

/* ------------------------------------------------------------------ Eqs. 6-8: per-pixel blend over the tile list */
typedef struct { int64_t vg; double alpha, T, G, raw, dx, dy; int clamped; } orc_contrib;

static double rel_gap(double x, double thr) { return fabs(x - thr) / fabs(thr); }

/* Blend one pixel; returns the number of contributors written to `out` (which must hold the tile list length).
 * near: bit 0 = a forward decision (alpha vs 1/255, T' vs 1e-4, exponent sign) lies within eps of its threshold,
 * bit 1 = alpha lies within eps of the 0.99 clamp. For alpha and T' the distance allowed also includes the rounding
 * a single-precision evaluation of the exponent -q0 - q1 - q2 can make when its terms cancel: its three terms each
 * carry about three roundings, and the base-2 exponential one more relative error, so 4 roundoffs of
 * mag = |q0| + |q1| + |q2| bound it (as a relative error of alpha = o e^power; times alpha / (1 - alpha) for T'). */
static int64_t blend_pixel(int W, double xs, double ys, const double *splat, const int64_t *list, int64_t lo,
                           int64_t hi, double eps, orc_contrib *out, double *T_final, int64_t *n_contrib,
                           int *near, double *rgb_acc)
{
    double T = 1.0;
    int64_t nc = 0, last = 0;
    *near = 0;
    rgb_acc[0] = rgb_acc[1] = rgb_acc[2] = 0.0;
    for (int64_t j = lo; j < hi; j++) {
        const double *sp = splat + 9 * list[j];
        double dx = sp[0] - xs, dy = sp[1] - ys;
        if (g_cam.model == 0) { /* minimal image across the longitude seam */
            if (dx >= 0.5 * W) dx -= W;
            else if (dx < -0.5 * W) dx += W;
        }
        double q0 = 0.5 * sp[2] * dx * dx, q2 = 0.5 * sp[4] * dy * dy, q1 = sp[3] * dx * dy;
        double power = -q0 - q2 - q1;
        double mag = fabs(q0) + fabs(q1) + fabs(q2);
        if (power > -eps * mag && mag > 0.0) *near |= 1;
        if (power > 0.0) continue;
        double G = exp(power);
        double raw = sp[5] * G;
        double cond = 4.0 * ORC_F32_ROUNDOFF * (mag + 1.0);
        if (rel_gap(raw, ORC_ALPHA_MIN) < eps + cond) *near |= 1;
        if (rel_gap(raw, ORC_ALPHA_MAX) < eps + cond) *near |= 2;
        int clamped = raw > ORC_ALPHA_MAX;
        double alpha = clamped ? ORC_ALPHA_MAX : raw;
        if (alpha < ORC_ALPHA_MIN) continue;
        double Tn = T * (1.0 - alpha);
        if (rel_gap(Tn, ORC_T_STOP) < eps + cond * alpha / (1.0 - alpha)) *near |= 1;
        if (Tn < ORC_T_STOP) break;
        for (int ch = 0; ch < 3; ch++) rgb_acc[ch] += sp[6 + ch] * alpha * T;
        out[nc].vg = list[j]; out[nc].alpha = alpha; out[nc].T = T; out[nc].G = G; out[nc].raw = raw;
        out[nc].dx = dx; out[nc].dy = dy; out[nc].clamped = clamped;
        nc++;
        T = Tn;
        last = j - lo + 1;
    }
    *T_final = T;
    *n_contrib = last;
    return nc;
}

/* splat: [V*n][9] = px, py, c0, c1, c2, opacity, r, g, b (conic c = Sigma~^-1 as (00, 01, 11)).
 * out_rgb [V,3,H,W], out_T [V,H,W], out_nc [V,H,W] (list position after the last contributor),
 * out_near [V,H,W] (see blend_pixel), out_count [V,H,W] (number of contributors; optional). */
void orc_blend_fwd(int V, int64_t n, int W, int H, int T, const double *bg, const double *splat,
                   const int64_t *ranges, const int64_t *list, double eps, double *out_rgb, double *out_T,
                   int32_t *out_nc, uint8_t *out_near, int32_t *out_count)
{
    int64_t TX = W / T, TY = H / T, tiles = TX * TY, maxlen = 1;
    (void)n;
    for (int64_t t = 0; t < V * tiles; t++)
        if (ranges[2 * t + 1] - ranges[2 * t] > maxlen) maxlen = ranges[2 * t + 1] - ranges[2 * t];
    orc_contrib *buf = (orc_contrib *)malloc(sizeof(orc_contrib) * maxlen);
    for (int v = 0; v < V; v++)
        for (int y = 0; y < H; y++)
            for (int x = 0; x < W; x++) {
                int64_t tile = v * tiles + (y / T) * TX + (x / T);
                double Tf, acc[3];
                int64_t nc;
                int near;
                int64_t count = blend_pixel(W, x + 0.5, y + 0.5, splat, list, ranges[2 * tile], ranges[2 * tile + 1],
                                            eps, buf, &Tf, &nc, &near, acc);
                int64_t pix = ((int64_t)v * H + y) * W + x;
                for (int ch = 0; ch < 3; ch++) out_rgb[((int64_t)v * 3 + ch) * H * W + (int64_t)y * W + x] = acc[ch] + Tf * bg[ch];
                out_T[pix] = Tf;
                out_nc[pix] = (int32_t)nc;
                out_near[pix] = (uint8_t)near;
                if (out_count) out_count[pix] = (int32_t)count;
            }
    free(buf);
}

/* Exact adjoint of orc_blend_fwd. grad: [V*n][G_LEN], overwritten. For contributor i of a pixel,
 *   dC/dc_i = a_i T_i,   dC/da_i = c_i T_i - (sum_{j>i} c_j a_j T_j + T_final bg) / (1 - a_i)
 * (T_i = prod_{j<i} (1 - a_j)), then through a = o G (unless clamped), G = exp(power) and
 * power = -1/2 (c0 dx^2 + c2 dy^2) - c1 dx dy with dx = p_x - x_s, dy = p_y - y_s. */
void orc_blend_bwd(int V, int64_t n, int W, int H, int T, const double *bg, const double *splat,
                   const int64_t *ranges, const int64_t *list, const double *dL_drgb, double *grad)
{
    int64_t TX = W / T, TY = H / T, tiles = TX * TY, maxlen = 1;
    for (int64_t t = 0; t < V * tiles; t++)
        if (ranges[2 * t + 1] - ranges[2 * t] > maxlen) maxlen = ranges[2 * t + 1] - ranges[2 * t];
    orc_contrib *buf = (orc_contrib *)malloc(sizeof(orc_contrib) * maxlen);
    double *suffix = (double *)malloc(sizeof(double) * 3 * (maxlen + 1));
    memset(grad, 0, sizeof(double) * G_LEN * V * n);
    for (int v = 0; v < V; v++)
        for (int y = 0; y < H; y++)
            for (int x = 0; x < W; x++) {
                int64_t tile = v * tiles + (y / T) * TX + (x / T);
                double Tf, acc[3], gC[3];
                int64_t ncpos;
                int near;
                int64_t nc = blend_pixel(W, x + 0.5, y + 0.5, splat, list, ranges[2 * tile], ranges[2 * tile + 1], 0.0,
                                         buf, &Tf, &ncpos, &near, acc);
                for (int ch = 0; ch < 3; ch++) gC[ch] = dL_drgb[((int64_t)v * 3 + ch) * H * W + (int64_t)y * W + x];
                /* suffix[i] = sum_{j>i} c_j a_j T_j + T_final bg */
                for (int ch = 0; ch < 3; ch++) suffix[3 * nc + ch] = Tf * bg[ch];
                for (int64_t i = nc - 1; i >= 0; i--) {
                    const double *sp = splat + 9 * buf[i].vg;
                    for (int ch = 0; ch < 3; ch++)
                        suffix[3 * i + ch] = suffix[3 * (i + 1) + ch] + sp[6 + ch] * buf[i].alpha * buf[i].T;
                }
                for (int64_t i = 0; i < nc; i++) {
                    const orc_contrib *c = &buf[i];
                    const double *sp = splat + 9 * c->vg;
                    double *gr = grad + G_LEN * c->vg;
                    double dL_dalpha = 0.0;
                    for (int ch = 0; ch < 3; ch++) {
                        gr[G_RED + ch] += c->alpha * c->T * gC[ch];
                        dL_dalpha += gC[ch] * (sp[6 + ch] * c->T - suffix[3 * (i + 1) + ch] / (1.0 - c->alpha));
                    }
                    if (c->clamped) continue;
                    gr[G_OPAC] += dL_dalpha * c->G;
                    double dL_dpower = dL_dalpha * sp[5] * c->G;
                    gr[G_C0] += -0.5 * c->dx * c->dx * dL_dpower;
                    gr[G_C1] += -c->dx * c->dy * dL_dpower;
                    gr[G_C2] += -0.5 * c->dy * c->dy * dL_dpower;
                    gr[G_PX] += (-sp[2] * c->dx - sp[3] * c->dy) * dL_dpower;
                    gr[G_PY] += (-sp[4] * c->dy - sp[3] * c->dx) * dL_dpower;
                }
            }
    free(buf);
    free(suffix);
}

/* ------------------------------------------------------------------ Eqs. 18-20: back to m, q, S, o, SH */
/* grad2d: [V*n][G_LEN] from orc_blend_bwd. Outputs are overwritten: d_means [n,3], d_scales [n,3],
 * d_quats [n,4], d_opacity [n], d_sh [n,K,3], d_screen [n,2] = dL/ds summed over views (p = (s + 1) (W, H) / 2). */
void orc_preprocess_bwd(int64_t n, int V, int W, int H, int sh_degree, double near_r,
                        const float *means, const float *scales, const float *quats, const float *opacity,
                        const float *sh, const float *viewmats, const double *grad2d,
                        double *d_means, double *d_scales, double *d_quats, double *d_opacity, double *d_sh,
                        double *d_screen)
{
    int K = (sh_degree + 1) * (sh_degree + 1);
    (void)opacity;
    memset(d_means, 0, sizeof(double) * 3 * n);
    memset(d_scales, 0, sizeof(double) * 3 * n);
    memset(d_quats, 0, sizeof(double) * 4 * n);
    memset(d_opacity, 0, sizeof(double) * n);
    memset(d_sh, 0, sizeof(double) * 3 * K * n);
    memset(d_screen, 0, sizeof(double) * 2 * n);
    for (int v = 0; v < V; v++) {
        double Wr[9], tcw[3], campos[3];
        load_view(viewmats + 16 * v, Wr, tcw, campos);
        for (int64_t g = 0; g < n; g++) {
            const double *gr = grad2d + (int64_t)G_LEN * (v * n + g);
            orc_fwd f;
            forward_one(W, H, sh_degree, near_r, means + 3 * g, scales + 3 * g, quats + 4 * g, sh + 3 * K * g,
                        opacity[g], Wr, tcw, campos, &f);
            if (f.culled) continue;
            double dt[3] = {0, 0, 0}, dm[3] = {0, 0, 0};
            /* opacity */
            d_opacity[g] += gr[G_OPAC];
            /* p(t): dp/dt (the Jacobian itself for the equirectangular camera, Eqs. 11-16) */
            for (int k = 0; k < 3; k++) dt[k] += gr[G_PX] * f.Jp[k] + gr[G_PY] * f.Jp[3 + k];
            d_screen[2 * g + 0] += gr[G_PX] * W / 2.0;
            d_screen[2 * g + 1] += gr[G_PY] * H / 2.0;
            /* conic = inverse of (a, b; b, c) */
            double a = f.cov[0], b = f.cov[1], c = f.cov[2], det = f.det, d2 = det * det;
            double gc0 = gr[G_C0], gc1 = gr[G_C1], gc2 = gr[G_C2];
            double dA = gc0 * (-c * c / d2) + gc1 * (b * c / d2) + gc2 * (-b * b / d2);
            double dB = gc0 * (2.0 * b * c / d2) + gc1 * (-(a * c + b * b) / d2) + gc2 * (2.0 * a * b / d2);
            double dC = gc0 * (-b * b / d2) + gc1 * (a * b / d2) + gc2 * (-a * a / d2);
            double G2[2][2] = {{dA, 0.5 * dB}, {0.5 * dB, dC}};
            /* Sigma~ = M Sigma M^T: dL/dSigma = M^T G2 M, dL/dM = 2 G2 M Sigma */
            double dSig[9], dM[6], MS[6];
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) {
                    double acc = 0.0;
                    for (int r = 0; r < 2; r++)
                        for (int s2 = 0; s2 < 2; s2++) acc += f.M[r * 3 + i] * G2[r][s2] * f.M[s2 * 3 + j];
                    dSig[i * 3 + j] = acc;
                }
            for (int r = 0; r < 2; r++)
                for (int j = 0; j < 3; j++) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; k++) acc += f.M[r * 3 + k] * f.Sig[k * 3 + j];
                    MS[r * 3 + j] = acc;
                }
            for (int r = 0; r < 2; r++)
                for (int j = 0; j < 3; j++) dM[r * 3 + j] = 2.0 * (G2[r][0] * MS[0 * 3 + j] + G2[r][1] * MS[1 * 3 + j]);
            /* M = J W: dL/dJ = dL/dM W^T */
            double dJ[6];
            for (int r = 0; r < 2; r++)
                for (int k = 0; k < 3; k++) {
                    double acc = 0.0;
                    for (int j = 0; j < 3; j++) acc += dM[r * 3 + j] * Wr[k * 3 + j];
                    dJ[r * 3 + k] = acc;
                }
            double dJdt[2][3][3];
            if (g_cam.model == 1) pinhole_jacobian_grad(f.t, W, H, dJdt);
            else jacobian_grad(f.t, W, H, dJdt);
            for (int r = 0; r < 2; r++)
                for (int cc = 0; cc < 3; cc++)
                    for (int k = 0; k < 3; k++) dt[k] += dJ[r * 3 + cc] * dJdt[r][cc][k];
            /* t = W m + t_cw */
            for (int j = 0; j < 3; j++) dm[j] += Wr[0 * 3 + j] * dt[0] + Wr[1 * 3 + j] * dt[1] + Wr[2 * 3 + j] * dt[2];
            /* Sigma = (R S)(R S)^T */
            double s[3] = {scales[3 * g], scales[3 * g + 1], scales[3 * g + 2]};
            double dR[9];
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) {
                    /* dL/d(RS)_ij = 2 (dSig (RS))_ij */
                    double acc = 0.0;
                    for (int k = 0; k < 3; k++) acc += dSig[i * 3 + k] * f.R[k * 3 + j] * s[j];
                    double dRS = 2.0 * acc;
                    dR[i * 3 + j] = dRS * s[j];
                    d_scales[3 * g + j] += dRS * f.R[i * 3 + j];
                }
            double qn[4], qv[4] = {quats[4 * g], quats[4 * g + 1], quats[4 * g + 2], quats[4 * g + 3]};
            double qnorm = sqrt(qv[0] * qv[0] + qv[1] * qv[1] + qv[2] * qv[2] + qv[3] * qv[3]);
            for (int k = 0; k < 4; k++) qn[k] = qv[k] / qnorm;
            double dRq[9][4], dqn[4] = {0, 0, 0, 0};
            rot_grad(qn, dRq);
            for (int e = 0; e < 9; e++)
                for (int k = 0; k < 4; k++) dqn[k] += dR[e] * dRq[e][k];
            double dot = dqn[0] * qn[0] + dqn[1] * qn[1] + dqn[2] * qn[2] + dqn[3] * qn[3];
            for (int k = 0; k < 4; k++) d_quats[4 * g + k] += (dqn[k] - qn[k] * dot) / qnorm;
            /* colour: c = max(sum_k Y_k(d) sh_k + 0.5, 0), d = (m - campos) / |m - campos| */
            double Y[16], dY[16][3], ddir[3] = {0, 0, 0};
            orc_sh_basis(sh_degree, f.dir, Y, &dY[0][0]);
            for (int ch = 0; ch < 3; ch++) {
                if (f.rgb_raw[ch] <= 0.0) continue;
                double gcol = gr[G_RED + ch];
                for (int k = 0; k < K; k++) {
                    d_sh[(3 * K) * g + 3 * k + ch] += Y[k] * gcol;
                    for (int j = 0; j < 3; j++) ddir[j] += sh[(3 * K) * g + 3 * k + ch] * dY[k][j] * gcol;
                }
            }
            double dd = ddir[0] * f.dir[0] + ddir[1] * f.dir[1] + ddir[2] * f.dir[2];
            for (int j = 0; j < 3; j++) dm[j] += (ddir[j] - f.dir[j] * dd) / f.dist;
            for (int j = 0; j < 3; j++) d_means[3 * g + j] += dm[j];
        }
    }
}
