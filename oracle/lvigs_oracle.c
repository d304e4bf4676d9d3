/*
 * lvigs_oracle.c -- plain, slow CPU oracle of the LVI-GS differentiable
 * Gaussian-splatting hot path (arxiv 2411.02703, Sec. III-B, III-D, III-E).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only tests/, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * Precision:
 *   - the "key stage" (view-space depth, screen position, radius, tile
 *     rectangle) is computed in strict IEEE binary32, one rounded operation at
 *     a time in the order written below (build with -ffp-contract=off), so the
 *     (tile, depth) keys can be compared bit for bit;
 *   - everything else (the values composited, the loss, every gradient) is
 *     computed in binary64 from the float inputs.
 *
 * Readings of the paper used here (the paper is silent on all of them):
 *   scale parameter is log-scale (s = exp), opacity parameter is a logit
 *   (o = sigmoid), quaternions are (w,x,y,z) normalised inside, the pose maps
 *   world -> camera with x right / y down / z forward, near plane 0.2,
 *   Jacobian clamp 1.3 * tan(half field of view), 0.3 px^2 dilation, radius
 *   ceil(3 sqrt(lambda_max)) with the eigenvalue discriminant floored at 0.1,
 *   pixel (px,py) is sampled at the integer coordinate, alpha clamp 0.99,
 *   1/255 cut-off, stop before a Gaussian that would drive T below 1e-4,
 *   d_i of Eq. (4) is view-space z, background black, real spherical
 *   harmonics (with the Condon-Shortley phase) plus 0.5 and clamped at 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_MEM 2

/* Camera (world -> camera rotation R row-major, translation t, pinhole). */
typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int W, H;
} orc_camera;

/* The key stage's scale: exp of the binary32 log-scale in binary64, rounded
 * once to binary32 (reading R1 of the scale activation). */
void orc_exp_key(const float *x, float *y, int64_t n) {
    for (int64_t i = 0; i < n; ++i) y[i] = (float)exp((double)x[i]);
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following oracle calls (for a single-core timing). */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Pyramid level camera (Sec. III-D): level l halves the image l times.      */
/* A level-l pixel covers a 2^l x 2^l block of level-0 pixels; with pixels   */
/* sampled at integer coordinates the block centre sits at 2^l p + (2^l-1)/2 */
/* so the principal point becomes (c + 0.5) / 2^l - 0.5.                     */
/* ------------------------------------------------------------------------ */
void orc_level_camera(const orc_camera *c0, int level, orc_camera *out) {
    float scale = 1.0f;
    for (int i = 0; i < level; ++i) scale = scale * 0.5f;
    *out = *c0;
    out->fx = c0->fx * scale;
    out->fy = c0->fy * scale;
    out->cx = (c0->cx + 0.5f) * scale - 0.5f;
    out->cy = (c0->cy + 0.5f) * scale - 0.5f;
    out->W = c0->W >> level;
    out->H = c0->H >> level;
}

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics up to degree 3 and their Cartesian gradients.    */
/* Y_{l,m} = sqrt(2) Re Y_l^m (m>0), Y_l^0 (m=0), sqrt(2) Im Y_l^|m| (m<0),  */
/* where Y_l^m carries the Condon-Shortley phase; index k = l^2 + l + m.     */
/* Written as polynomials of the unit direction (x, y, z).                   */
/* ------------------------------------------------------------------------ */
static void sh_basis(double x, double y, double z, double Y[16], double dY[16][3]) {
    const double PI = 3.14159265358979323846;
    const double k0 = 0.5 / sqrt(PI);
    const double k1 = sqrt(3.0 / (4.0 * PI));
    const double k2a = 0.5 * sqrt(15.0 / PI);
    const double k2b = 0.25 * sqrt(5.0 / PI);
    const double k2c = 0.25 * sqrt(15.0 / PI);
    const double k3a = 0.25 * sqrt(35.0 / (2.0 * PI));
    const double k3b = 0.5 * sqrt(105.0 / PI);
    const double k3c = 0.25 * sqrt(21.0 / (2.0 * PI));
    const double k3d = 0.25 * sqrt(7.0 / PI);
    const double k3e = 0.25 * sqrt(105.0 / PI);
    double xx = x * x, yy = y * y, zz = z * z;
    memset(dY, 0, sizeof(double) * 48);
    /* l = 0 */
    Y[0] = k0;
    /* l = 1: m = -1, 0, 1 */
    Y[1] = -k1 * y;            dY[1][1] = -k1;
    Y[2] = k1 * z;             dY[2][2] = k1;
    Y[3] = -k1 * x;            dY[3][0] = -k1;
    /* l = 2 */
    Y[4] = k2a * x * y;        dY[4][0] = k2a * y; dY[4][1] = k2a * x;
    Y[5] = -k2a * y * z;       dY[5][1] = -k2a * z; dY[5][2] = -k2a * y;
    Y[6] = k2b * (2 * zz - xx - yy);
    dY[6][0] = -2 * k2b * x; dY[6][1] = -2 * k2b * y; dY[6][2] = 4 * k2b * z;
    Y[7] = -k2a * x * z;       dY[7][0] = -k2a * z; dY[7][2] = -k2a * x;
    Y[8] = k2c * (xx - yy);    dY[8][0] = 2 * k2c * x; dY[8][1] = -2 * k2c * y;
    /* l = 3 */
    Y[9] = -k3a * y * (3 * xx - yy);
    dY[9][0] = -k3a * 6 * x * y; dY[9][1] = -k3a * (3 * xx - 3 * yy);
    Y[10] = k3b * x * y * z;
    dY[10][0] = k3b * y * z; dY[10][1] = k3b * x * z; dY[10][2] = k3b * x * y;
    Y[11] = -k3c * y * (4 * zz - xx - yy);
    dY[11][0] = -k3c * (-2 * x * y); dY[11][1] = -k3c * (4 * zz - xx - 3 * yy);
    dY[11][2] = -k3c * 8 * y * z;
    Y[12] = k3d * z * (2 * zz - 3 * xx - 3 * yy);
    dY[12][0] = k3d * (-6 * x * z); dY[12][1] = k3d * (-6 * y * z);
    dY[12][2] = k3d * (6 * zz - 3 * xx - 3 * yy);
    Y[13] = -k3c * x * (4 * zz - xx - yy);
    dY[13][0] = -k3c * (4 * zz - 3 * xx - yy); dY[13][1] = -k3c * (-2 * x * y);
    dY[13][2] = -k3c * 8 * x * z;
    Y[14] = k3e * z * (xx - yy);
    dY[14][0] = k3e * 2 * x * z; dY[14][1] = -k3e * 2 * y * z; dY[14][2] = k3e * (xx - yy);
    Y[15] = -k3a * x * (xx - 3 * yy);
    dY[15][0] = -k3a * (3 * xx - 3 * yy); dY[15][1] = -k3a * (-6 * x * y);
}

/* Exported for the orthonormality / library pins. */
void orc_sh_basis(double x, double y, double z, double *Y16, double *dY48) {
    double Y[16], dY[16][3];
    sh_basis(x, y, z, Y, dY);
    memcpy(Y16, Y, sizeof Y);
    if (dY48) memcpy(dY48, dY, sizeof dY);
}

/* ------------------------------------------------------------------------ */
/* Key stage, strict binary32 (Eq. (2) and Eq. (7) up to the radius).       */
/* Each statement is one rounded IEEE operation; the order is the contract.  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int visible;         /* 0: culled (behind the near plane or singular)  */
    float z;             /* view-space depth, the low half of the key      */
    float u, v;          /* screen position                                */
    float a, b, c, det;  /* dilated 2D covariance and its determinant      */
    int radius;          /* ceil(3 sqrt(lambda_max))                       */
    int x0, y0, x1, y1;  /* covered tile rectangle, [x0,x1) x [y0,y1)      */
} key_stage_t;

static float clamp_tile(float f, int hi) {
    if (!(f > 0.0f)) return 0.0f;
    if (f > (float)hi) return (float)hi;
    return f;
}

static void key_stage(const float *m, const float *ls, const float *q, const orc_camera *c,
                      int tw, int th, int tiles_x, int tiles_y, key_stage_t *o) {
    const float *R = c->R;
    memset(o, 0, sizeof *o);
    /* mu_I = [Q_iw, T_iw] mu_W  (Eq. 7) */
    float px = R[0] * m[0]; px = px + R[1] * m[1]; px = px + R[2] * m[2]; px = px + c->t[0];
    float py = R[3] * m[0]; py = py + R[4] * m[1]; py = py + R[5] * m[2]; py = py + c->t[1];
    float pz = R[6] * m[0]; pz = pz + R[7] * m[1]; pz = pz + R[8] * m[2]; pz = pz + c->t[2];
    if (!(pz > 0.2f)) return;
    /* S = diag(exp(log_scale)); exp evaluated in binary64 and rounded once */
    float s0 = (float)exp((double)ls[0]);
    float s1 = (float)exp((double)ls[1]);
    float s2 = (float)exp((double)ls[2]);
    /* unit quaternion (w, x, y, z) */
    float n2 = q[0] * q[0]; n2 = n2 + q[1] * q[1]; n2 = n2 + q[2] * q[2]; n2 = n2 + q[3] * q[3];
    if (!(n2 > 0.0f)) return;
    float nr = sqrtf(n2);
    float w = q[0] / nr, x = q[1] / nr, y = q[2] / nr, z = q[3] / nr;
    float r[9];
    r[0] = 1.0f - 2.0f * (y * y + z * z);
    r[1] = 2.0f * (x * y - w * z);
    r[2] = 2.0f * (x * z + w * y);
    r[3] = 2.0f * (x * y + w * z);
    r[4] = 1.0f - 2.0f * (x * x + z * z);
    r[5] = 2.0f * (y * z - w * x);
    r[6] = 2.0f * (x * z - w * y);
    r[7] = 2.0f * (y * z + w * x);
    r[8] = 1.0f - 2.0f * (x * x + y * y);
    /* M = R S, Sigma = M M^T  (Eq. 2) */
    float M[9];
    M[0] = r[0] * s0; M[1] = r[1] * s1; M[2] = r[2] * s2;
    M[3] = r[3] * s0; M[4] = r[4] * s1; M[5] = r[5] * s2;
    M[6] = r[6] * s0; M[7] = r[7] * s1; M[8] = r[8] * s2;
    float S[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            float acc = M[3 * i] * M[3 * j];
            acc = acc + M[3 * i + 1] * M[3 * j + 1];
            acc = acc + M[3 * i + 2] * M[3 * j + 2];
            S[3 * i + j] = acc;
        }
    /* linearised projection J with the field-of-view clamp */
    float xz = px / pz, yz = py / pz;
    float limx = 1.3f * ((0.5f * (float)c->W) / c->fx);
    float limy = 1.3f * ((0.5f * (float)c->H) / c->fy);
    float txc = xz < -limx ? -limx : (xz > limx ? limx : xz);
    float tyc = yz < -limy ? -limy : (yz > limy ? limy : yz);
    float J00 = c->fx / pz;
    float J02 = -(c->fx * txc) / pz;
    float J11 = c->fy / pz;
    float J12 = -(c->fy * tyc) / pz;
    /* T = J Q_iw; Sigma_I = T Sigma T^T  (Eq. 7) */
    float T[6];
    for (int j = 0; j < 3; ++j) {
        T[j] = J00 * R[j] + J02 * R[6 + j];
        T[3 + j] = J11 * R[3 + j] + J12 * R[6 + j];
    }
    float U[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            float acc = T[3 * i] * S[j];
            acc = acc + T[3 * i + 1] * S[3 + j];
            acc = acc + T[3 * i + 2] * S[6 + j];
            U[3 * i + j] = acc;
        }
    float a = U[0] * T[0]; a = a + U[1] * T[1]; a = a + U[2] * T[2];
    float b = U[0] * T[3]; b = b + U[1] * T[4]; b = b + U[2] * T[5];
    float cc = U[3] * T[3]; cc = cc + U[4] * T[4]; cc = cc + U[5] * T[5];
    a = a + 0.3f;
    cc = cc + 0.3f;
    float det = a * cc - b * b;
    if (!(det > 0.0f)) return;
    float mid = 0.5f * (a + cc);
    float disc = mid * mid - det;
    float lam = mid + sqrtf(disc > 0.1f ? disc : 0.1f);
    int rad = (int)ceilf(3.0f * sqrtf(lam));
    float u = c->fx * xz + c->cx;
    float v = c->fy * yz + c->cy;
    float fr = (float)rad;
    o->visible = 1;
    o->z = pz;
    o->u = u;
    o->v = v;
    o->a = a;
    o->b = b;
    o->c = cc;
    o->det = det;
    o->radius = rad;
    o->x0 = (int)clamp_tile((u - fr) / (float)tw, tiles_x);
    o->x1 = (int)clamp_tile((u + fr + (float)(tw - 1)) / (float)tw, tiles_x);
    o->y0 = (int)clamp_tile((v - fr) / (float)th, tiles_y);
    o->y1 = (int)clamp_tile((v + fr + (float)(th - 1)) / (float)th, tiles_y);
}

/* ------------------------------------------------------------------------ */
/* Binary64 per-Gaussian values (Eq. 2, Eq. 6 opacity, Eq. 7, SH colour).    */
/* ------------------------------------------------------------------------ */
typedef struct {
    double p[3];          /* view-space mean                        */
    double s[3];          /* scales                                 */
    double qn[4], qnorm;  /* unit quaternion and |q|                 */
    double r[9];          /* rotation of the quaternion             */
    double Sig[9];        /* 3D covariance                          */
    double J[4];          /* J00, J02, J11, J12                     */
    int clampx, clampy;   /* J used the clamped tangent             */
    double T[6];          /* J Q_iw                                 */
    double a, b, c;       /* dilated 2D covariance                  */
    double det;
    double conic[3];      /* A, B, C of the inverse                 */
    double u, v;          /* screen position                        */
    double opacity;       /* sigmoid(logit)                         */
    double dir[3], dirlen, dirn[3];
    double Y[16], dY[16][3];
    double rgb_raw[3], rgb[3];
    double rgb_margin;    /* min over channels of |rgb_raw| / (0.5 + sum |sh Y|) */
} g64_t;

static void value_stage(const float *m, const float *ls, const float *q, float ol, const float *sh,
                        int K, int deg, const orc_camera *c, g64_t *g) {
    const float *R = c->R;
    double Rd[9], td[3];
    for (int i = 0; i < 9; ++i) Rd[i] = R[i];
    for (int i = 0; i < 3; ++i) td[i] = c->t[i];
    double fx = c->fx, fy = c->fy, cx = c->cx, cy = c->cy;
    for (int i = 0; i < 3; ++i)
        g->p[i] = Rd[3 * i] * m[0] + Rd[3 * i + 1] * m[1] + Rd[3 * i + 2] * m[2] + td[i];
    for (int i = 0; i < 3; ++i) g->s[i] = exp((double)ls[i]);
    double qq[4] = {q[0], q[1], q[2], q[3]};
    g->qnorm = sqrt(qq[0] * qq[0] + qq[1] * qq[1] + qq[2] * qq[2] + qq[3] * qq[3]);
    for (int i = 0; i < 4; ++i) g->qn[i] = qq[i] / g->qnorm;
    double w = g->qn[0], x = g->qn[1], y = g->qn[2], z = g->qn[3];
    double *r = g->r;
    r[0] = 1 - 2 * (y * y + z * z); r[1] = 2 * (x * y - w * z); r[2] = 2 * (x * z + w * y);
    r[3] = 2 * (x * y + w * z); r[4] = 1 - 2 * (x * x + z * z); r[5] = 2 * (y * z - w * x);
    r[6] = 2 * (x * z - w * y); r[7] = 2 * (y * z + w * x); r[8] = 1 - 2 * (x * x + y * y);
    /* Sigma = R S S^T R^T */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += r[3 * i + k] * g->s[k] * g->s[k] * r[3 * j + k];
            g->Sig[3 * i + j] = acc;
        }
    double pz = g->p[2];
    double xz = g->p[0] / pz, yz = g->p[1] / pz;
    double limx = 1.3 * (0.5 * c->W / fx), limy = 1.3 * (0.5 * c->H / fy);
    double txc = xz, tyc = yz;
    g->clampx = g->clampy = 0;
    if (xz < -limx) { txc = -limx; g->clampx = 1; }
    if (xz > limx) { txc = limx; g->clampx = 1; }
    if (yz < -limy) { tyc = -limy; g->clampy = 1; }
    if (yz > limy) { tyc = limy; g->clampy = 1; }
    g->J[0] = fx / pz;
    g->J[1] = -fx * txc / pz;
    g->J[2] = fy / pz;
    g->J[3] = -fy * tyc / pz;
    for (int j = 0; j < 3; ++j) {
        g->T[j] = g->J[0] * Rd[j] + g->J[1] * Rd[6 + j];
        g->T[3 + j] = g->J[2] * Rd[3 + j] + g->J[3] * Rd[6 + j];
    }
    double a = 0, b = 0, cc = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            a += g->T[i] * g->Sig[3 * i + j] * g->T[j];
            b += g->T[i] * g->Sig[3 * i + j] * g->T[3 + j];
            cc += g->T[3 + i] * g->Sig[3 * i + j] * g->T[3 + j];
        }
    g->a = a + 0.3;
    g->b = b;
    g->c = cc + 0.3;
    g->det = g->a * g->c - g->b * g->b;
    g->conic[0] = g->c / g->det;
    g->conic[1] = -g->b / g->det;
    g->conic[2] = g->a / g->det;
    g->u = fx * xz + cx;
    g->v = fy * yz + cy;
    g->opacity = 1.0 / (1.0 + exp(-(double)ol));
    /* view direction from the camera centre C = -R^T t to the mean */
    double C[3];
    for (int i = 0; i < 3; ++i) C[i] = -(Rd[i] * td[0] + Rd[3 + i] * td[1] + Rd[6 + i] * td[2]);
    for (int i = 0; i < 3; ++i) g->dir[i] = (double)m[i] - C[i];
    g->dirlen = sqrt(g->dir[0] * g->dir[0] + g->dir[1] * g->dir[1] + g->dir[2] * g->dir[2]);
    for (int i = 0; i < 3; ++i) g->dirn[i] = g->dir[i] / g->dirlen;
    sh_basis(g->dirn[0], g->dirn[1], g->dirn[2], g->Y, g->dY);
    int nk = (deg + 1) * (deg + 1);
    g->rgb_margin = INFINITY;
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0, mag = 0.5;
        for (int k = 0; k < nk; ++k) {
            acc += (double)sh[k * 3 + ch] * g->Y[k];
            mag += fabs((double)sh[k * 3 + ch] * g->Y[k]);
        }
        g->rgb_raw[ch] = acc + 0.5;
        g->rgb[ch] = g->rgb_raw[ch] < 0 ? 0 : g->rgb_raw[ch];
        const double m = fabs(g->rgb_raw[ch]) / mag;
        if (m < g->rgb_margin) g->rgb_margin = m;
    }
    (void)K;
}

/* ------------------------------------------------------------------------ */
/* a1: preprocess one view.                                                  */
/* Key outputs (float/int): z, u, v, radius, rect[4], tiles_touched.         */
/* Value outputs (double):  uv[2], conic[3], opacity, rgb[3], depth.         */
/* screen_key selects which screen-space Gaussian the values describe:      */
/*   1  the key stage's own: its binary32 centre (u, v) and depth z, and the  */
/*      binary64 inverse of its binary32 covariance (the same projection,    */
/*      Eq. 7, that decides the tile lists; the paper's pipeline computes it */
/*      once, in binary32);                                                  */
/*   0  the projection recomputed in binary64 (a smooth function of the      */
/*      parameters, for finite-difference checks of the gradients).          */
/* Opacity and colour are binary64 in both.                                  */
/* rgb_margin (optional): distance of the SH colour's clamp at 0, relative to */
/* the magnitude of its terms (min over channels; INFINITY when culled).      */
/* conic_f[3] (optional): the inverse of the key stage's binary32 covariance */
/* (its binary32 a, b, c over its binary32 determinant), taken in binary64:  */
/* the conic a binary32 compositing stage starts from, for the error         */
/* allowance of the render margins.                                          */
/* ------------------------------------------------------------------------ */
int orc_preprocess(int64_t n, const float *means, const float *log_scales, const float *quats,
                   const float *opacity_logits, const float *sh, int sh_stride_k, int sh_degree,
                   const orc_camera *cam, int tile_w, int tile_h,
                   float *z_f, float *uv_f, int32_t *radius, int32_t *rect, uint32_t *tiles,
                   double *uv, double *conic, double *opacity, double *rgb, double *depth,
                   double *conic_f, double *rgb_margin, int screen_key) {
    if (n < 0 || tile_w <= 0 || tile_h <= 0 || sh_degree < 0 || sh_degree > 3 ||
        sh_stride_k < (sh_degree + 1) * (sh_degree + 1))
        return ORC_ERR_ARG;
    int tiles_x = (cam->W + tile_w - 1) / tile_w;
    int tiles_y = (cam->H + tile_h - 1) / tile_h;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        key_stage_t k;
        key_stage(means + 3 * i, log_scales + 3 * i, quats + 4 * i, cam, tile_w, tile_h, tiles_x,
                  tiles_y, &k);
        z_f[i] = k.z;
        uv_f[2 * i] = k.u;
        uv_f[2 * i + 1] = k.v;
        radius[i] = k.visible ? k.radius : 0;
        rect[4 * i] = k.x0; rect[4 * i + 1] = k.y0; rect[4 * i + 2] = k.x1; rect[4 * i + 3] = k.y1;
        tiles[i] = k.visible ? (uint32_t)((k.x1 - k.x0) * (k.y1 - k.y0)) : 0u;
        if (conic_f) {
            if (k.visible) {
                conic_f[3 * i] = (double)k.c / (double)k.det;
                conic_f[3 * i + 1] = -(double)k.b / (double)k.det;
                conic_f[3 * i + 2] = (double)k.a / (double)k.det;
            } else {
                conic_f[3 * i] = conic_f[3 * i + 1] = conic_f[3 * i + 2] = 0;
            }
        }
        if (rgb_margin) rgb_margin[i] = INFINITY;
        if (!k.visible) {
            uv[2 * i] = uv[2 * i + 1] = 0;
            conic[3 * i] = conic[3 * i + 1] = conic[3 * i + 2] = 0;
            opacity[i] = 0; rgb[3 * i] = rgb[3 * i + 1] = rgb[3 * i + 2] = 0; depth[i] = 0;
            continue;
        }
        g64_t g;
        value_stage(means + 3 * i, log_scales + 3 * i, quats + 4 * i, opacity_logits[i],
                    sh + (size_t)i * sh_stride_k * 3, sh_stride_k, sh_degree, cam, &g);
        if (screen_key) {
            uv[2 * i] = (double)k.u; uv[2 * i + 1] = (double)k.v;
            conic[3 * i] = (double)k.c / (double)k.det;
            conic[3 * i + 1] = -(double)k.b / (double)k.det;
            conic[3 * i + 2] = (double)k.a / (double)k.det;
            depth[i] = (double)k.z;
        } else {
            uv[2 * i] = g.u; uv[2 * i + 1] = g.v;
            conic[3 * i] = g.conic[0]; conic[3 * i + 1] = g.conic[1]; conic[3 * i + 2] = g.conic[2];
            depth[i] = g.p[2];
        }
        opacity[i] = g.opacity;
        for (int ch = 0; ch < 3; ++ch) rgb[3 * i + ch] = g.rgb[ch];
        if (rgb_margin) rgb_margin[i] = g.rgb_margin;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* a2 + a3: (tile, depth) keys, sorted.  key = (tile_base + ty*tiles_x + tx) */
/* << 32 | bits(z); value = Gaussian index.  Sorted by (key, value), which   */
/* is the unique stable order of the emission sequence.                     */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t key; uint32_t val; } kv_t;

static int kv_cmp(const void *pa, const void *pb) {
    const kv_t *a = (const kv_t *)pa, *b = (const kv_t *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->val != b->val) return a->val < b->val ? -1 : 1;
    return 0;
}

int64_t orc_count_instances(int64_t n, const uint32_t *tiles) {
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) m += tiles[i];
    return m;
}

int orc_build_keys(int64_t n, const int32_t *rect, const float *z_f, const uint32_t *tiles,
                   int tiles_x, uint32_t tile_base, int64_t m_cap, uint64_t *keys, uint32_t *vals) {
    int64_t m = orc_count_instances(n, tiles);
    if (m > m_cap) return ORC_ERR_ARG;
    kv_t *kv = (kv_t *)malloc(sizeof(kv_t) * (size_t)(m > 0 ? m : 1));
    if (!kv) return ORC_ERR_MEM;
    int64_t w = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (tiles[i] == 0) continue;
        uint32_t zb;
        memcpy(&zb, &z_f[i], 4);
        for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ++ty)
            for (int tx = rect[4 * i]; tx < rect[4 * i + 2]; ++tx) {
                uint64_t tile = (uint64_t)tile_base + (uint64_t)ty * (uint64_t)tiles_x + (uint64_t)tx;
                kv[w].key = (tile << 32) | (uint64_t)zb;
                kv[w].val = (uint32_t)i;
                ++w;
            }
    }
    qsort(kv, (size_t)m, sizeof(kv_t), kv_cmp);
    for (int64_t j = 0; j < m; ++j) { keys[j] = kv[j].key; vals[j] = kv[j].val; }
    free(kv);
    return ORC_OK;
}

/* a4: per-tile [start, end) of the sorted instance list. */
int orc_tile_ranges(int64_t m, const uint64_t *keys, uint32_t tile_base, int n_tiles,
                    uint32_t *ranges) {
    for (int t = 0; t < n_tiles; ++t) ranges[2 * t] = ranges[2 * t + 1] = 0;
    for (int64_t j = 0; j < m; ++j) {
        int64_t t = (int64_t)(keys[j] >> 32) - (int64_t)tile_base;
        if (t < 0 || t >= n_tiles) continue;
        if (j == 0 || (keys[j - 1] >> 32) != (keys[j] >> 32)) ranges[2 * t] = (uint32_t)j;
        ranges[2 * t + 1] = (uint32_t)(j + 1);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* a5: front-to-back compositing (Eq. 3, 4, 5, 6) of a pixel over its tile's */
/* sorted list.  One walk serves both the images and their gradients, so the */
/* two take the same decisions.                                              */
/*                                                                           */
/* Per Gaussian, in list order: power = -(A dx^2 + C dy^2)/2 - B dx dy       */
/* (skipped if positive), alpha = min(0.99, o e^power) (Eq. 6), skipped if   */
/* alpha < 1/255, and the walk stops before a Gaussian that would take T     */
/* below 1e-4.                                                               */
/*                                                                           */
/* The walk also reports the smallest relative distance ("margin") of any    */
/* test to its threshold, so callers can tell pixels where binary32          */
/* arithmetic may legitimately take the other branch.  With uv_f / conic_f   */
/* (the binary32 centre of the key stage and the conic of its binary32       */
/* covariance) the distance of each test on alpha, o G and T is net of an    */
/* allowance for binary32: the exponent moves by                             */
/*   d_in  = |power(uv_f, conic_f) - power(uv, conic)|                       */
/* (the deviation the binary32 inputs force, evaluated in binary64; zero     */
/* when the values already are the key stage's) plus                         */
/*   d_ev  = 16 u (scale + |ln o| + 1),  u = 2^-24,                          */
/* for the rounding of evaluating it in binary32 (the conic from the         */
/* covariance, the offsets, products and sums, the logarithm of the binary32 */
/* opacity) and of the exponential, and alpha and o G move by the same       */
/* amount relatively (first order).  T's relative allowance grows by         */
/* alpha / (1 - alpha) times that, plus 2 u, per blended Gaussian.  The      */
/* power > 0 test can only go the other way at binary64 rounding, where a    */
/* binary32 evaluation has no such test at all: its margin is 0 when |power| */
/* is within 64 binary64 ulps of the terms' scale and does not count         */
/* otherwise.                                                                */
/*                                                                           */
/* "close" tests are those whose margin is at most close_margin.  With       */
/* flip = 1 every close test takes the other branch: the result is the other */
/* outcome the same arithmetic may legitimately give (first order: every     */
/* close call at once).                                                      */
/* ------------------------------------------------------------------------ */
#define ALPHA_MAX 0.99
#define ALPHA_MIN (1.0 / 255.0)
#define T_MIN 1e-4

static double rel_margin(double x, double thr) { return fabs(x - thr) / fabs(thr); }

#define U32 (1.0 / 16777216.0)
#define U64 (1.0 / 9007199254740992.0)

typedef struct {
    uint32_t g;
    uint32_t pos;          /* position in the tile's list */
    double alpha, T, G, dx, dy;
    int clamped;
} contrib_t;

typedef struct {
    const double *uv, *conic, *opacity;
    const float *uv_f;     /* optional: allowance of the binary32 inputs */
    const double *conic_f;
    double close_margin;   /* tests with margin <= this are close */
    int flip;              /* close tests take the other branch */
} walk_in;

typedef struct {
    contrib_t *lst;        /* contributors in list order (grown on demand) */
    size_t cap, cnt;
    double T, margin;
    int32_t last, nclose;
    uint64_t sig;          /* FNV-1a of the contributing positions */
} walk_out;

/* Walk one pixel over vals[s, e).  Returns 0, or 1 if memory ran out. */
static int walk_pixel(const walk_in *in, const uint32_t *vals, uint32_t s, uint32_t e, int px,
                      int py, walk_out *w) {
    const int allow = in->uv_f && in->conic_f;
    double T = 1.0, margin = INFINITY, eT = 0; /* eT: relative allowance of T */
    int32_t last = 0, nclose = 0;
    uint64_t sig = 1469598103934665603ull;
    w->cnt = 0;
    for (uint32_t j = s; j < e; ++j) {
        uint32_t g = vals[j];
        double dx = in->uv[2 * g] - px, dy = in->uv[2 * g + 1] - py;
        double A = in->conic[3 * g], B = in->conic[3 * g + 1], Cc = in->conic[3 * g + 2];
        double power = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy;
        double scale = 0.5 * (fabs(A) * dx * dx + fabs(Cc) * dy * dy) + fabs(B * dx * dy);
        double o = in->opacity[g];
        /* power > 0: only at binary64 rounding */
        int skip_pos = power > 0;
        if (scale > 0 && fabs(power) <= 64.0 * U64 * scale) {
            if (0.0 < margin) margin = 0.0;
            if (0.0 <= in->close_margin) {
                ++nclose;
                if (in->flip) skip_pos = !skip_pos;
            }
        }
        if (skip_pos) continue;
        double da = 16.0 * U32 * (scale + fabs(log(o)) + 1.0); /* relative allowance of o G, alpha */
        if (allow) {
            double fx = (double)in->uv_f[2 * g] - px, fy = (double)in->uv_f[2 * g + 1] - py;
            double Af = in->conic_f[3 * g], Bf = in->conic_f[3 * g + 1], Cf = in->conic_f[3 * g + 2];
            double pf = -0.5 * (Af * fx * fx + Cf * fy * fy) - Bf * fx * fy;
            da += fabs(pf - power);
        }
        double G = exp(power);
        double oG = o * G;
        /* the 0.99 clamp */
        int clamped = !(oG < ALPHA_MAX);
        double mc = rel_margin(oG, ALPHA_MAX) - da;
        if (mc < margin) margin = mc;
        if (mc <= in->close_margin) {
            ++nclose;
            if (in->flip) clamped = !clamped;
        }
        double alpha = clamped ? ALPHA_MAX : oG;
        /* the 1/255 cut */
        int take = alpha >= ALPHA_MIN;
        double ma = rel_margin(alpha, ALPHA_MIN) - da;
        if (ma < margin) margin = ma;
        if (ma <= in->close_margin) {
            ++nclose;
            if (in->flip) take = !take;
        }
        if (!take) continue;
        /* the 1e-4 stop */
        double Tn = T * (1.0 - alpha);
        eT += alpha / (1.0 - alpha) * da + 2.0 * U32;
        int stop = Tn < T_MIN;
        double mt = rel_margin(Tn, T_MIN) - eT;
        if (mt < margin) margin = mt;
        if (mt <= in->close_margin) {
            ++nclose;
            if (in->flip) stop = !stop;
        }
        if (stop) break;
        if (w->cnt == w->cap) {
            size_t nc = w->cap ? 2 * w->cap : 64;
            contrib_t *nl = (contrib_t *)realloc(w->lst, sizeof(contrib_t) * nc);
            if (!nl) return 1;
            w->lst = nl;
            w->cap = nc;
        }
        contrib_t *c = &w->lst[w->cnt++];
        c->g = g; c->pos = j - s; c->alpha = alpha; c->T = T; c->G = G; c->dx = dx; c->dy = dy;
        c->clamped = clamped;
        T = Tn;
        last = (int32_t)(j - s + 1);
        sig = (sig ^ (uint64_t)(j - s)) * 1099511628211ull;
    }
    w->T = T;
    w->margin = margin;
    w->last = last;
    w->nclose = nclose;
    w->sig = sig;
    return 0;
}

int orc_render(int W, int H, int tile_w, int tile_h, const double *uv, const double *conic,
               const double *opacity, const double *rgb, const double *depth,
               const uint32_t *vals, const uint32_t *ranges, int n_sel, const int32_t *sel_tiles,
               double *out_rgb, double *out_depth, double *out_alpha, double *out_T,
               int32_t *out_ncontrib, double *out_margin, uint64_t *out_sig,
               const float *uv_f, const double *conic_f, double close_margin, int flip,
               int32_t *out_nclose) {
    int tiles_x = (W + tile_w - 1) / tile_w;
    int tiles_y = (H + tile_h - 1) / tile_h;
    int nt = sel_tiles ? n_sel : tiles_x * tiles_y;
    walk_in in = {uv, conic, opacity, uv_f, conic_f, close_margin, flip};
    int err = 0;
#pragma omp parallel
    {
        walk_out w;
        memset(&w, 0, sizeof w);
#pragma omp for schedule(dynamic, 1)
        for (int it = 0; it < nt; ++it) {
            int t = sel_tiles ? sel_tiles[it] : it;
            if (t < 0 || t >= tiles_x * tiles_y) continue;
            int tx = t % tiles_x, ty = t / tiles_x;
            uint32_t s = ranges[2 * t], e = ranges[2 * t + 1];
            for (int py = ty * tile_h; py < (ty + 1) * tile_h && py < H; ++py)
                for (int px = tx * tile_w; px < (tx + 1) * tile_w && px < W; ++px) {
                    if (walk_pixel(&in, vals, s, e, px, py, &w)) {
#pragma omp atomic write
                        err = 1;
                        continue;
                    }
                    /* Eq. (3), (4): sums of x_i alpha_i T_i; Eq. (5): V = 1 - T */
                    double C[3] = {0, 0, 0}, D = 0;
                    for (size_t i = 0; i < w.cnt; ++i) {
                        const contrib_t *c = &w.lst[i];
                        double wgt = c->alpha * c->T;
                        for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * c->g + ch] * wgt;
                        D += depth[c->g] * wgt;
                    }
                    size_t p = (size_t)py * W + px;
                    if (out_sig) out_sig[p] = w.sig;
                    for (int ch = 0; ch < 3; ++ch) out_rgb[(size_t)ch * W * H + p] = C[ch];
                    out_depth[p] = D;
                    out_alpha[p] = 1.0 - w.T;
                    out_T[p] = w.T;
                    out_ncontrib[p] = w.last;
                    if (out_margin) out_margin[p] = w.margin;
                    if (out_nclose) out_nclose[p] = w.nclose;
                }
        }
        free(w.lst);
    }
    return err ? ORC_ERR_MEM : ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* a6: gradient of the composited images with respect to each Gaussian's     */
/* screen-space values.  For pixel p with contributing list 1..n, weights    */
/* w_i = alpha_i T_i and T_i = prod_{j<i}(1-alpha_j):                        */
/*   dX/dalpha_i = x_i T_i - (1/(1-alpha_i)) sum_{k>i} x_k w_k   (X = C,D)   */
/*   dV/dalpha_i = T_i     - (1/(1-alpha_i)) sum_{k>i} w_k                   */
/*   dX/dx_i     = w_i                                                       */
/* then alpha_i = o_i exp(power_i) with power as in Eq. (6).                */
/* Output per Gaussian (10 doubles): du, dv, dA, dB, dC, dopacity,           */
/* drgb[3], ddepth.  The walk (and its close_margin / flip) is the one of    */
/* orc_render.                                                               */
/* ------------------------------------------------------------------------ */
int orc_backward_render(int W, int H, int tile_w, int tile_h, int64_t n, const double *uv,
                        const double *conic, const double *opacity, const double *rgb,
                        const double *depth, const uint32_t *vals, const uint32_t *ranges,
                        const double *dL_drgb, const double *dL_ddepth, const double *dL_dalpha,
                        double *grad2d, const float *uv_f, const double *conic_f,
                        double close_margin, int flip) {
    int tiles_x = (W + tile_w - 1) / tile_w;
    int tiles_y = (H + tile_h - 1) / tile_h;
    int nt = tiles_x * tiles_y;
    int nthr = orc_num_threads();
    double *acc = (double *)calloc((size_t)nthr * (size_t)n * 10, sizeof(double));
    if (!acc) return ORC_ERR_MEM;
    walk_in in = {uv, conic, opacity, uv_f, conic_f, close_margin, flip};
    int err = 0;
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *my = acc + (size_t)tid * (size_t)n * 10;
        walk_out w;
        memset(&w, 0, sizeof w);
        size_t scap = 0;
        double *suf = NULL;
#pragma omp for schedule(dynamic, 1)
        for (int t = 0; t < nt; ++t) {
            int tx = t % tiles_x, ty = t / tiles_x;
            uint32_t s = ranges[2 * t], e = ranges[2 * t + 1];
            for (int py = ty * tile_h; py < (ty + 1) * tile_h && py < H; ++py)
                for (int px = tx * tile_w; px < (tx + 1) * tile_w && px < W; ++px) {
                    size_t p = (size_t)py * W + px;
                    if (walk_pixel(&in, vals, s, e, px, py, &w)) {
#pragma omp atomic write
                        err = 1;
                        continue;
                    }
                    size_t cnt = w.cnt;
                    if (cnt + 1 > scap) {
                        double *ns = (double *)realloc(suf, sizeof(double) * 5 * (cnt + 1));
                        if (!ns) {
#pragma omp atomic write
                            err = 1;
                            continue;
                        }
                        suf = ns;
                        scap = cnt + 1;
                    }
                    const contrib_t *lst = w.lst;
                    /* suffix sums of x_k w_k for x in (r, g, b, depth, 1) */
                    for (int q = 0; q < 5; ++q) suf[5 * cnt + q] = 0;
                    for (size_t i = cnt; i-- > 0;) {
                        const contrib_t *c = &lst[i];
                        double wgt = c->alpha * c->T;
                        suf[5 * i + 0] = suf[5 * (i + 1) + 0] + rgb[3 * c->g + 0] * wgt;
                        suf[5 * i + 1] = suf[5 * (i + 1) + 1] + rgb[3 * c->g + 1] * wgt;
                        suf[5 * i + 2] = suf[5 * (i + 1) + 2] + rgb[3 * c->g + 2] * wgt;
                        suf[5 * i + 3] = suf[5 * (i + 1) + 3] + depth[c->g] * wgt;
                        suf[5 * i + 4] = suf[5 * (i + 1) + 4] + wgt;
                    }
                    double gc[3];
                    for (int ch = 0; ch < 3; ++ch) gc[ch] = dL_drgb[(size_t)ch * W * H + p];
                    double gd = dL_ddepth ? dL_ddepth[p] : 0.0;
                    double ga = dL_dalpha ? dL_dalpha[p] : 0.0;
                    for (size_t i = 0; i < cnt; ++i) {
                        const contrib_t *c = &lst[i];
                        uint32_t g = c->g;
                        double wgt = c->alpha * c->T;
                        double inv = 1.0 / (1.0 - c->alpha);
                        double dLda = 0;
                        for (int ch = 0; ch < 3; ++ch)
                            dLda += gc[ch] * (rgb[3 * g + ch] * c->T - suf[5 * (i + 1) + ch] * inv);
                        dLda += gd * (depth[g] * c->T - suf[5 * (i + 1) + 3] * inv);
                        dLda += ga * (c->T - suf[5 * (i + 1) + 4] * inv);
                        double *o = my + (size_t)g * 10;
                        for (int ch = 0; ch < 3; ++ch) o[6 + ch] += gc[ch] * wgt;
                        o[9] += gd * wgt;
                        if (c->clamped) continue;
                        double A = conic[3 * g], B = conic[3 * g + 1], Cc = conic[3 * g + 2];
                        double dLdpow = dLda * c->alpha;
                        o[5] += dLda * c->G;
                        o[0] += dLdpow * (-(A * c->dx + B * c->dy));
                        o[1] += dLdpow * (-(Cc * c->dy + B * c->dx));
                        o[2] += dLdpow * (-0.5 * c->dx * c->dx);
                        o[3] += dLdpow * (-c->dx * c->dy);
                        o[4] += dLdpow * (-0.5 * c->dy * c->dy);
                    }
                }
        }
        free(w.lst);
        free(suf);
    }
    for (int64_t i = 0; i < n * 10; ++i) {
        double sacc = 0;
        for (int th = 0; th < nthr; ++th) sacc += acc[(size_t)th * (size_t)n * 10 + i];
        grad2d[i] = sacc;
    }
    free(acc);
    return err ? ORC_ERR_MEM : ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* a7: chain rule from the screen-space gradients to the parameters          */
/* (Eq. 2, Eq. 7, sigmoid opacity, SH colour).  Adds into the outputs so     */
/* several views accumulate.                                                  */
/* ------------------------------------------------------------------------ */
int orc_backward_preprocess(int64_t n, const float *means, const float *log_scales,
                            const float *quats, const float *opacity_logits, const float *sh,
                            int sh_stride_k, int sh_degree, const orc_camera *cam,
                            const uint32_t *tiles, const double *grad2d,
                            double *d_means, double *d_log_scales, double *d_quats,
                            double *d_opacity_logits, double *d_sh) {
    const int K = sh_stride_k;
    int nk = (sh_degree + 1) * (sh_degree + 1);
    double Rd[9];
    for (int i = 0; i < 9; ++i) Rd[i] = cam->R[i];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        if (tiles[i] == 0) continue;
        const double *g2 = grad2d + (size_t)i * 10;
        int any = 0;
        for (int k = 0; k < 10; ++k) any |= g2[k] != 0.0;
        if (!any) continue;
        g64_t g;
        value_stage(means + 3 * i, log_scales + 3 * i, quats + 4 * i, opacity_logits[i],
                    sh + (size_t)i * K * 3, K, sh_degree, cam, &g);
        double du = g2[0], dv = g2[1], dA = g2[2], dB = g2[3], dC = g2[4];
        double dop = g2[5], dz = g2[9];
        double dmean[3] = {0, 0, 0};
        /* opacity = sigmoid(logit) */
        d_opacity_logits[i] += dop * g.opacity * (1.0 - g.opacity);
        /* colour: rgb = max(0, sum_k sh_k Y_k(dir) + 0.5) */
        double ddirn[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ++ch) {
            if (g.rgb_raw[ch] < 0) continue;
            double dc = g2[6 + ch];
            for (int k = 0; k < nk; ++k) {
                d_sh[((size_t)i * K + k) * 3 + ch] += dc * g.Y[k];
                for (int a = 0; a < 3; ++a) ddirn[a] += dc * (double)sh[((size_t)i * K + k) * 3 + ch] * g.dY[k][a];
            }
        }
        /* dirn = dir / |dir|, dir = mean - C */
        double dd = ddirn[0] * g.dirn[0] + ddirn[1] * g.dirn[1] + ddirn[2] * g.dirn[2];
        for (int a = 0; a < 3; ++a) dmean[a] += (ddirn[a] - g.dirn[a] * dd) / g.dirlen;
        /* conic = inverse of [[a, b], [b, c]] */
        double a = g.a, b = g.b, c = g.c, det = g.det, det2 = det * det;
        double da = dA * (-c * c / det2) + dB * (b * c / det2) + dC * (1.0 / det - a * c / det2);
        double dc_ = dA * (1.0 / det - a * c / det2) + dB * (a * b / det2) + dC * (-a * a / det2);
        double db = dA * (2.0 * b * c / det2) + dB * (-1.0 / det - 2.0 * b * b / det2) + dC * (2.0 * a * b / det2);
        /* 2D covariance entries: a = T0 Sig T0^T, b = T0 Sig T1^T, c = T1 Sig T1^T */
        double dSig[9];
        for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s)
                dSig[3 * r + s] = da * g.T[r] * g.T[s] + db * g.T[r] * g.T[3 + s] + dc_ * g.T[3 + r] * g.T[3 + s];
        double dT[6];
        for (int r = 0; r < 3; ++r) {
            double s0 = 0, s1 = 0;
            for (int s = 0; s < 3; ++s) { s0 += g.Sig[3 * r + s] * g.T[s]; s1 += g.Sig[3 * r + s] * g.T[3 + s]; }
            dT[r] = 2.0 * da * s0 + db * s1;
            dT[3 + r] = db * s0 + 2.0 * dc_ * s1;
        }
        /* T = J Q_iw: T0j = J00 R0j + J02 R2j, T1j = J11 R1j + J12 R2j */
        double dJ00 = 0, dJ02 = 0, dJ11 = 0, dJ12 = 0;
        for (int j = 0; j < 3; ++j) {
            dJ00 += dT[j] * Rd[j];
            dJ02 += dT[j] * Rd[6 + j];
            dJ11 += dT[3 + j] * Rd[3 + j];
            dJ12 += dT[3 + j] * Rd[6 + j];
        }
        double fx = cam->fx, fy = cam->fy;
        double px = g.p[0], py = g.p[1], pz = g.p[2];
        double dp[3] = {0, 0, 0};
        /* J00 = fx/pz, J11 = fy/pz */
        dp[2] += dJ00 * (-fx / (pz * pz)) + dJ11 * (-fy / (pz * pz));
        /* J02 = -fx txc / pz with txc = px/pz unless clamped */
        if (g.clampx) {
            double txc = -g.J[1] * pz / fx;
            dp[2] += dJ02 * (fx * txc / (pz * pz));
        } else {
            dp[0] += dJ02 * (-fx / (pz * pz));
            dp[2] += dJ02 * (2.0 * fx * px / (pz * pz * pz));
        }
        if (g.clampy) {
            double tyc = -g.J[3] * pz / fy;
            dp[2] += dJ12 * (fy * tyc / (pz * pz));
        } else {
            dp[1] += dJ12 * (-fy / (pz * pz));
            dp[2] += dJ12 * (2.0 * fy * py / (pz * pz * pz));
        }
        /* u = fx px/pz + cx, v = fy py/pz + cy, depth = pz */
        dp[0] += du * fx / pz;
        dp[1] += dv * fy / pz;
        dp[2] += du * (-fx * px / (pz * pz)) + dv * (-fy * py / (pz * pz)) + dz;
        /* p = Q_iw mean + T_iw */
        for (int a2 = 0; a2 < 3; ++a2)
            dmean[a2] += Rd[a2] * dp[0] + Rd[3 + a2] * dp[1] + Rd[6 + a2] * dp[2];
        /* Sigma = (R S)(R S)^T: dM = (dSig + dSig^T) M, M = R diag(s) */
        double M[9], dM[9];
        for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s) M[3 * r + s] = g.r[3 * r + s] * g.s[s];
        for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += (dSig[3 * r + k] + dSig[3 * k + r]) * M[3 * k + s];
                dM[3 * r + s] = acc;
            }
        double dR[9];
        for (int s = 0; s < 3; ++s) {
            double dsv = 0;
            for (int r = 0; r < 3; ++r) { dsv += dM[3 * r + s] * g.r[3 * r + s]; dR[3 * r + s] = dM[3 * r + s] * g.s[s]; }
            d_log_scales[3 * i + s] += dsv * g.s[s];
        }
        double w = g.qn[0], x = g.qn[1], y = g.qn[2], z = g.qn[3];
        double dqn[4];
        dqn[0] = 2 * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
        dqn[1] = 2 * (y * dR[1] + z * dR[2] + y * dR[3] - 2 * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] - 2 * x * dR[8]);
        dqn[2] = 2 * (-2 * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] - 2 * y * dR[8]);
        dqn[3] = 2 * (-2 * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2 * z * dR[4] + y * dR[5] + x * dR[6] + y * dR[7]);
        double dot = dqn[0] * g.qn[0] + dqn[1] * g.qn[1] + dqn[2] * g.qn[2] + dqn[3] * g.qn[3];
        for (int k = 0; k < 4; ++k) d_quats[4 * i + k] += (dqn[k] - g.qn[k] * dot) / g.qnorm;
        for (int a2 = 0; a2 < 3; ++a2) d_means[3 * i + a2] += dmean[a2];
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* a8: L = (1-lambda) L1 + lambda (1 - mean SSIM) + lambda_d L_d             */
/* (Eq. 10, 11, 12).  SSIM: 11x11 Gaussian window (sigma 1.5, normalised),   */
/* zero padding, C1 = 0.01^2, C2 = 0.03^2, mean over channels and pixels.    */
/* L_d: mean |D - D_lidar| over pixels with D_lidar > 0 (0 if none).         */
/* Gradients with sign(0) = 0.  With flip = 1 an L1 residual within          */
/* kink_margin (colour) or depth_kink_margin (depth) of zero takes the other */
/* sign: the subgradient a residual that small may legitimately get when the */
/* image is known only to that tolerance.                                    */
/* ------------------------------------------------------------------------ */
static void ssim_window(double w[11]) {
    double s = 0;
    for (int i = 0; i < 11; ++i) { w[i] = exp(-((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5)); s += w[i]; }
    for (int i = 0; i < 11; ++i) w[i] /= s;
}

static double sgn(double x) { return x > 0 ? 1.0 : (x < 0 ? -1.0 : 0.0); }

static double sgn_flip(double x, double margin, int flip) {
    return (flip && fabs(x) <= margin) ? -sgn(x) : sgn(x);
}

int orc_loss(int W, int H, const double *img, const double *gt, const double *depth,
             const double *lidar, double lambda, double lambda_d, double *loss_terms,
             double *d_img, double *d_depth, double kink_margin, double depth_kink_margin,
             int flip) {
    size_t P = (size_t)W * H;
    double w1[11];
    ssim_window(w1);
    double l1 = 0;
    for (size_t i = 0; i < 3 * P; ++i) {
        l1 += fabs(img[i] - gt[i]);
        if (d_img) d_img[i] = (1.0 - lambda) * sgn_flip(img[i] - gt[i], kink_margin, flip) / (3.0 * P);
    }
    l1 /= (3.0 * P);
    double ssim_mean = 0;
    if (lambda != 0.0) {
        const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
        double *G1 = (double *)malloc(sizeof(double) * P);
        double *G2 = (double *)malloc(sizeof(double) * P);
        double *G12 = (double *)malloc(sizeof(double) * P);
        if (!G1 || !G2 || !G12) { free(G1); free(G2); free(G12); return ORC_ERR_MEM; }
        for (int ch = 0; ch < 3; ++ch) {
            const double *x = img + ch * P, *y = gt + ch * P;
            double csum = 0;
#pragma omp parallel for schedule(static) reduction(+ : csum)
            for (int py = 0; py < H; ++py)
                for (int px = 0; px < W; ++px) {
                    double mx = 0, my = 0, mxx = 0, myy = 0, mxy = 0;
                    for (int i = -5; i <= 5; ++i)
                        for (int j = -5; j <= 5; ++j) {
                            int qy = py + i, qx = px + j;
                            if (qy < 0 || qy >= H || qx < 0 || qx >= W) continue;
                            double wt = w1[i + 5] * w1[j + 5];
                            double xv = x[(size_t)qy * W + qx], yv = y[(size_t)qy * W + qx];
                            mx += wt * xv; my += wt * yv;
                            mxx += wt * xv * xv; myy += wt * yv * yv; mxy += wt * xv * yv;
                        }
                    double sx = mxx - mx * mx, sy = myy - my * my, sxy = mxy - mx * my;
                    double A1 = 2 * mx * my + C1, A2 = 2 * sxy + C2;
                    double B1 = mx * mx + my * my + C1, B2 = sx + sy + C2;
                    double S = (A1 * A2) / (B1 * B2);
                    csum += S;
                    size_t p = (size_t)py * W + px;
                    /* partial derivatives of S w.r.t. the raw moments mx, mxx, mxy */
                    G1[p] = (2 * my * A2 - 2 * my * A1) / (B1 * B2) - S * (2 * mx / B1 - 2 * mx / B2);
                    G2[p] = -S / B2;
                    G12[p] = 2 * A1 / (B1 * B2);
                }
            ssim_mean += csum;
            if (d_img) {
                double kfac = -lambda / (3.0 * P);
#pragma omp parallel for schedule(static)
                for (int qy = 0; qy < H; ++qy)
                    for (int qx = 0; qx < W; ++qx) {
                        double s1 = 0, s2 = 0, s12 = 0;
                        for (int i = -5; i <= 5; ++i)
                            for (int j = -5; j <= 5; ++j) {
                                int py = qy + i, px = qx + j;
                                if (py < 0 || py >= H || px < 0 || px >= W) continue;
                                double wt = w1[i + 5] * w1[j + 5];
                                size_t p = (size_t)py * W + px;
                                s1 += wt * G1[p]; s2 += wt * G2[p]; s12 += wt * G12[p];
                            }
                        size_t q = (size_t)qy * W + qx;
                        d_img[ch * P + q] += kfac * (s1 + 2.0 * x[q] * s2 + y[q] * s12);
                    }
            }
        }
        ssim_mean /= (3.0 * P);
        free(G1); free(G2); free(G12);
    }
    double ld = 0;
    size_t nvalid = 0;
    for (size_t i = 0; i < P; ++i) if (lidar[i] > 0) ++nvalid;
    for (size_t i = 0; i < P; ++i) {
        if (d_depth) d_depth[i] = 0;
        if (!(lidar[i] > 0)) continue;
        ld += fabs(depth[i] - lidar[i]);
        if (d_depth)
            d_depth[i] = lambda_d * sgn_flip(depth[i] - lidar[i], depth_kink_margin, flip) / (double)nvalid;
    }
    if (nvalid) ld /= (double)nvalid;
    double loss = (1.0 - lambda) * l1 + (lambda != 0.0 ? lambda * (1.0 - ssim_mean) : 0.0) + lambda_d * ld;
    if (loss_terms) {
        loss_terms[0] = loss;
        loss_terms[1] = l1;
        loss_terms[2] = lambda != 0.0 ? ssim_mean : 1.0;
        loss_terms[3] = ld;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* a9: one pyramid level down (Sec. III-D): RGB 2x2 box mean; depth = mean   */
/* of the valid (> 0) samples of the 2x2 block, else 0.                       */
/* ------------------------------------------------------------------------ */
int orc_pyramid_down(int W, int H, const double *rgb, const double *depth, double *rgb_out,
                     double *depth_out) {
    int W2 = W / 2, H2 = H / 2;
    for (int ch = 0; ch < 3; ++ch)
        for (int y = 0; y < H2; ++y)
            for (int x = 0; x < W2; ++x) {
                const double *s = rgb + (size_t)ch * W * H;
                double a = s[(size_t)(2 * y) * W + 2 * x] + s[(size_t)(2 * y) * W + 2 * x + 1] +
                           s[(size_t)(2 * y + 1) * W + 2 * x] + s[(size_t)(2 * y + 1) * W + 2 * x + 1];
                rgb_out[(size_t)ch * W2 * H2 + (size_t)y * W2 + x] = 0.25 * a;
            }
    for (int y = 0; y < H2; ++y)
        for (int x = 0; x < W2; ++x) {
            double sum = 0;
            int cnt = 0;
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    double d = depth[(size_t)(2 * y + dy) * W + 2 * x + dx];
                    if (d > 0) { sum += d; ++cnt; }
                }
            depth_out[(size_t)y * W2 + x] = cnt ? sum / cnt : 0.0;
        }
    return ORC_OK;
}
