/*
 * lsv2_oracle.c -- plain, single-threaded FP64 CPU oracle for sparse-coefficient
 * Gaussian splatting (LangSplatV2, arXiv 2507.07136).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file; only the tests, the package smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, constant table or helper with
 * the CUDA path: the two are written separately from the same equations.
 *
 * What it computes, in the paper's order:
 *   - Sec. 3.1, Eq. 1-2 and EWA splatting: each Gaussian's 2D mean and the
 *     inverse ("conic") of its projected, dilated 2D covariance (FP64).
 *   - The tile binning and depth order of Eq. 3's "ordered Gaussian points within
 *     a tile": one instance per (Gaussian, tile of its screen rectangle), ordered
 *     by (tile, depth, id).  The integer decisions (visibility, radius, rectangle,
 *     depth key) follow an FP32 decision specification so they can be compared
 *     bit for bit; near-degenerate Gaussians take those decisions in FP64.
 *   - Eq. 3 front-to-back alpha blending with the weights e_i of Eq. 7, and
 *     Algorithm 1's sparse accumulation W[j] += w_ij * e_i over the K pairs.
 *     Two more accumulation modes exist to state Sec. 3.3/3.4's identities:
 *     dense L-vector coefficients ("blending zeros does not alter the result")
 *     and dense D-dim features f_i = w_i S (Eq. 6), equal by Eq. 7 to W S.
 *   - Eq. 7 decode F = W S, and the relevancy score of Sec. 3.2 (cosine
 *     similarity, min over canonical negatives of the pairwise softmax).
 *   - The gradient of the blend with respect to the per-Gaussian quantities,
 *     written as the literal derivative of Eq. 3/7 (an O(n^2) sum per pixel),
 *     and the projection's Jacobian by complex-step differentiation of the same
 *     FP64 projection code (exact to rounding).
 *
 * Readings where the paper is silent (constants of the 3DGS rasteriser that the
 * paper builds on): dilation 0.3 px^2 on the 2D covariance, screen radius
 * ceil(3 sqrt(lambda_max)), guard band 1.3 tan(fov/2) on the Jacobian, near
 * plane 0.2, alpha clamp 0.99, skip alpha < 1/255, stop before a Gaussian that
 * would drive T below 1e-4.  All thresholds are the float32 values of these
 * constants, widened exactly to double.
 *
 * Compile: gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC (no FMA
 * contraction: the FP32 decision path relies on every float op being rounded).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_DILATION_F 0.3f
#define ORC_GUARD_F 1.3f
#define ORC_DEGENERATE_COND_F 1e6f
#define ORC_DISC_FLOOR_F 0.1f
#define ORC_RADIUS_CAP_F 1048576.0f
#define ORC_ALPHA_MAX ((double)0.99f)
#define ORC_ALPHA_MIN ((double)(1.0f / 255.0f))
#define ORC_T_MIN ((double)1e-4f)

typedef struct {
    int32_t width, height, tile_w, tile_h;
    float fx, fy, cx, cy, near_z;
    float R[9]; /* world->camera rotation, row-major */
    float t[3]; /* world->camera translation */
} orc_camera;

typedef double complex cplx;

static int32_t grid_x(const orc_camera* c) { return (c->width + c->tile_w - 1) / c->tile_w; }
static int32_t grid_y(const orc_camera* c) { return (c->height + c->tile_h - 1) / c->tile_h; }

/* ======================================================================================
 * 1. FP32 decision path.  Every float operation is correctly rounded and evaluated in
 *    the order written (no contraction).  Produces visibility, the degenerate flag,
 *    the integer radius, the tile rectangle [x0,x1) x [y0,y1) and the depth key.
 * ==================================================================================== */

static int32_t clamp_floor_to_int(float f, int32_t lo, int32_t hi)
{
    if (!(f >= (float)lo)) return lo; /* also catches NaN */
    if (f > (float)hi) return hi;
    return (int32_t)f;
}

typedef struct {
    int visible, degenerate;
    int32_t radius, x0, y0, x1, y1;
    float depth_key;
} decision;

/* Quaternion (w,x,y,z), already normalised, to the rotation matrix (standard form). */
static void rot_from_unit_quat_f(float w, float x, float y, float z, float R[9])
{
    R[0] = 1.0f - 2.0f * (y * y + z * z);
    R[1] = 2.0f * (x * y - w * z);
    R[2] = 2.0f * (x * z + w * y);
    R[3] = 2.0f * (x * y + w * z);
    R[4] = 1.0f - 2.0f * (x * x + z * z);
    R[5] = 2.0f * (y * z - w * x);
    R[6] = 2.0f * (x * z - w * y);
    R[7] = 2.0f * (y * z + w * x);
    R[8] = 1.0f - 2.0f * (x * x + y * y);
}

static void rot_from_unit_quat_d(double w, double x, double y, double z, double R[9])
{
    R[0] = 1.0 - 2.0 * (y * y + z * z);
    R[1] = 2.0 * (x * y - w * z);
    R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);
    R[4] = 1.0 - 2.0 * (x * x + z * z);
    R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);
    R[7] = 2.0 * (y * z + w * x);
    R[8] = 1.0 - 2.0 * (x * x + y * y);
}

/* FP64 re-evaluation of the covariance part of the decision path for near-degenerate
 * Gaussians: the same steps in double from the exactly widened float inputs.  Returns
 * the radius and writes the depth key (t_z rounded to float). */
static int32_t degenerate_radius_f64(const orc_camera* c, const float* m, const float* s,
                                     const float* q, float* depth_key)
{
    double Rv[9], tv[3];
    for (int i = 0; i < 9; ++i) Rv[i] = (double)c->R[i];
    for (int i = 0; i < 3; ++i) tv[i] = (double)c->t[i];
    double t[3];
    for (int i = 0; i < 3; ++i)
        t[i] = ((Rv[3 * i + 0] * (double)m[0] + Rv[3 * i + 1] * (double)m[1]) +
                Rv[3 * i + 2] * (double)m[2]) + tv[i];
    double qw = q[0], qx = q[1], qy = q[2], qz = q[3];
    double n2 = ((qw * qw + qx * qx) + qy * qy) + qz * qz;
    double inv = 1.0 / sqrt(n2);
    double R[9];
    rot_from_unit_quat_d(qw * inv, qx * inv, qy * inv, qz * inv, R);
    double M[9];
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j) M[3 * k + j] = R[3 * k + j] * (double)s[j];
    double tanx = (double)c->width / (2.0 * (double)c->fx);
    double tany = (double)c->height / (2.0 * (double)c->fy);
    double limx = (double)ORC_GUARD_F * tanx, limy = (double)ORC_GUARD_F * tany;
    double txz = t[0] / t[2], tyz = t[1] / t[2];
    double cxz = fmin(limx, fmax(-limx, txz)), cyz = fmin(limy, fmax(-limy, tyz));
    double J00 = (double)c->fx / t[2], J11 = (double)c->fy / t[2];
    double J02 = -((double)c->fx * cxz) / t[2], J12 = -((double)c->fy * cyz) / t[2];
    double T[6];
    for (int j = 0; j < 3; ++j) {
        T[j] = J00 * Rv[j] + J02 * Rv[6 + j];
        T[3 + j] = J11 * Rv[3 + j] + J12 * Rv[6 + j];
    }
    double N[6];
    for (int a = 0; a < 2; ++a)
        for (int j = 0; j < 3; ++j)
            N[3 * a + j] = (T[3 * a + 0] * M[j] + T[3 * a + 1] * M[3 + j]) + T[3 * a + 2] * M[6 + j];
    double s00 = (N[0] * N[0] + N[1] * N[1]) + N[2] * N[2];
    double s11 = (N[3] * N[3] + N[4] * N[4]) + N[5] * N[5];
    double s01 = (N[0] * N[3] + N[1] * N[4]) + N[2] * N[5];
    double d = (double)ORC_DILATION_F;
    double mid = 0.5 * ((s00 + d) + (s11 + d));
    double hd = 0.5 * (s00 - s11);
    double disc = fmax((double)ORC_DISC_FLOOR_F, hd * hd + s01 * s01);
    double lam = mid + sqrt(disc);
    double rf = ceil(3.0 * sqrt(lam));
    if (!(rf < (double)ORC_RADIUS_CAP_F)) rf = (double)ORC_RADIUS_CAP_F;
    *depth_key = (float)t[2];
    return (int32_t)rf;
}

static decision decide(const orc_camera* c, const float* m, const float* s, const float* q)
{
    decision o;
    memset(&o, 0, sizeof(o));
    const float* Rv = c->R;
    float t0 = ((Rv[0] * m[0] + Rv[1] * m[1]) + Rv[2] * m[2]) + c->t[0];
    float t1 = ((Rv[3] * m[0] + Rv[4] * m[1]) + Rv[5] * m[2]) + c->t[1];
    float t2 = ((Rv[6] * m[0] + Rv[7] * m[1]) + Rv[8] * m[2]) + c->t[2];
    if (!(t2 > c->near_z)) return o;
    float n2 = ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3];
    if (!(n2 > 0.0f)) return o;
    float inv = 1.0f / sqrtf(n2);
    float R[9];
    rot_from_unit_quat_f(q[0] * inv, q[1] * inv, q[2] * inv, q[3] * inv, R);
    float M[9];
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j) M[3 * k + j] = R[3 * k + j] * s[j];
    float tanx = (float)c->width / (2.0f * c->fx);
    float tany = (float)c->height / (2.0f * c->fy);
    float limx = ORC_GUARD_F * tanx, limy = ORC_GUARD_F * tany;
    float txz = t0 / t2, tyz = t1 / t2;
    float cxz = fminf(limx, fmaxf(-limx, txz)), cyz = fminf(limy, fmaxf(-limy, tyz));
    float J00 = c->fx / t2, J11 = c->fy / t2;
    float J02 = -(c->fx * cxz) / t2, J12 = -(c->fy * cyz) / t2;
    float T[6];
    for (int j = 0; j < 3; ++j) {
        T[j] = J00 * Rv[j] + J02 * Rv[6 + j];
        T[3 + j] = J11 * Rv[3 + j] + J12 * Rv[6 + j];
    }
    float N[6];
    for (int a = 0; a < 2; ++a)
        for (int j = 0; j < 3; ++j)
            N[3 * a + j] = (T[3 * a + 0] * M[j] + T[3 * a + 1] * M[3 + j]) + T[3 * a + 2] * M[6 + j];
    float s00 = (N[0] * N[0] + N[1] * N[1]) + N[2] * N[2];
    float s11 = (N[3] * N[3] + N[4] * N[4]) + N[5] * N[5];
    float s01 = (N[0] * N[3] + N[1] * N[4]) + N[2] * N[5];
    float k0 = N[1] * N[5] - N[2] * N[4];
    float k1 = N[2] * N[3] - N[0] * N[5];
    float k2 = N[0] * N[4] - N[1] * N[3];
    float det0 = (k0 * k0 + k1 * k1) + k2 * k2;
    float tr = s00 + s11;
    o.degenerate = !(det0 * ORC_DEGENERATE_COND_F > tr * tr);
    int32_t radius;
    if (!o.degenerate) {
        float d = ORC_DILATION_F;
        float mid = 0.5f * ((s00 + d) + (s11 + d));
        float hd = 0.5f * (s00 - s11);
        float disc = fmaxf(ORC_DISC_FLOOR_F, hd * hd + s01 * s01);
        float lam = mid + sqrtf(disc);
        float rf = ceilf(3.0f * sqrtf(lam));
        if (!(rf < ORC_RADIUS_CAP_F)) rf = ORC_RADIUS_CAP_F;
        radius = (int32_t)rf;
        o.depth_key = t2;
    } else {
        radius = degenerate_radius_f64(c, m, s, q, &o.depth_key);
    }
    float u = c->fx * txz + c->cx;
    float v = c->fy * tyz + c->cy;
    float r = (float)radius;
    float tw = (float)c->tile_w, th = (float)c->tile_h;
    int32_t GX = grid_x(c), GY = grid_y(c);
    o.x0 = clamp_floor_to_int(floorf((u - r) / tw), 0, GX);
    o.x1 = clamp_floor_to_int(floorf(((u + r) + (tw - 1.0f)) / tw), 0, GX);
    o.y0 = clamp_floor_to_int(floorf((v - r) / th), 0, GY);
    o.y1 = clamp_floor_to_int(floorf(((v + r) + (th - 1.0f)) / th), 0, GY);
    o.radius = radius;
    o.visible = (o.x1 > o.x0) && (o.y1 > o.y0);
    return o;
}

/* ======================================================================================
 * 2. FP64 projection (Eq. 1-2, EWA).  Written over complex numbers so that complex-step
 *    differentiation gives the exact Jacobian for the gradient oracle; with real inputs
 *    all imaginary parts stay zero.  Inputs: mean m[3], scale s[3], quaternion q[4]
 *    (normalised here).  Outputs: 2D mean (u, v) and conic (a, b, c) = inverse of the
 *    dilated 2D covariance [[c00, c01], [c01, c11]].
 * ==================================================================================== */

static cplx cmin_re(cplx a, cplx b) { return creal(a) <= creal(b) ? a : b; }
static cplx cmax_re(cplx a, cplx b) { return creal(a) >= creal(b) ? a : b; }

static void project_c(const orc_camera* c, const cplx* m, const cplx* s, const cplx* q,
                      cplx* uv, cplx* conic, cplx* cov)
{
    cplx Rv[9], t[3];
    for (int i = 0; i < 9; ++i) Rv[i] = (double)c->R[i];
    for (int i = 0; i < 3; ++i) t[i] = Rv[3 * i] * m[0] + Rv[3 * i + 1] * m[1] + Rv[3 * i + 2] * m[2] + (double)c->t[i];
    /* unit quaternion -> rotation R (Eq. 2) */
    cplx qn = csqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    cplx w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
    cplx R[9] = {1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y),
                 2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x),
                 2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)};
    /* Sigma = R S S^T R^T with S = diag(s) (Eq. 2) */
    cplx Sig[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx acc = 0;
            for (int k = 0; k < 3; ++k) acc += R[3 * i + k] * s[k] * s[k] * R[3 * j + k];
            Sig[3 * i + j] = acc;
        }
    /* camera-space covariance W Sigma W^T */
    cplx Sc[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx acc = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) acc += Rv[3 * i + a] * Sig[3 * a + b] * Rv[3 * j + b];
            Sc[3 * i + j] = acc;
        }
    /* EWA: local affine approximation J of the perspective projection, guard-band clamp */
    double tanx = (double)c->width / (2.0 * (double)c->fx);
    double tany = (double)c->height / (2.0 * (double)c->fy);
    double limx = (double)ORC_GUARD_F * tanx, limy = (double)ORC_GUARD_F * tany;
    cplx txz = t[0] / t[2], tyz = t[1] / t[2];
    cplx cx_ = cmin_re(limx, cmax_re(-limx, txz)) * t[2];
    cplx cy_ = cmin_re(limy, cmax_re(-limy, tyz)) * t[2];
    double fx = c->fx, fy = c->fy;
    cplx J[6] = {fx / t[2], 0.0, -fx * cx_ / (t[2] * t[2]), 0.0, fy / t[2], -fy * cy_ / (t[2] * t[2])};
    cplx S2[4];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            cplx acc = 0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) acc += J[3 * a + i] * Sc[3 * i + j] * J[3 * b + j];
            S2[2 * a + b] = acc;
        }
    double d = (double)ORC_DILATION_F;
    cplx c00 = S2[0] + d, c01 = 0.5 * (S2[1] + S2[2]), c11 = S2[3] + d;
    cplx det = c00 * c11 - c01 * c01;
    conic[0] = c11 / det;
    conic[1] = -c01 / det;
    conic[2] = c00 / det;
    if (cov) { cov[0] = c00; cov[1] = c01; cov[2] = c11; }
    uv[0] = fx * t[0] / t[2] + (double)c->cx;
    uv[1] = fy * t[1] / t[2] + (double)c->cy;
}

static void project_d(const orc_camera* c, const double* m, const double* s, const double* q,
                      double* uv, double* conic, double* cov)
{
    cplx mc[3], sc[3], qc[4], uvc[2], cc[3], vc[3];
    for (int i = 0; i < 3; ++i) { mc[i] = m[i]; sc[i] = s[i]; }
    for (int i = 0; i < 4; ++i) qc[i] = q[i];
    project_c(c, mc, sc, qc, uvc, cc, vc);
    uv[0] = creal(uvc[0]); uv[1] = creal(uvc[1]);
    for (int i = 0; i < 3; ++i) conic[i] = creal(cc[i]);
    if (cov) for (int i = 0; i < 3; ++i) cov[i] = creal(vc[i]);
}

/* Public: project n Gaussians.  Decision outputs (bit-exact spec) and FP64 values. */
void orc_project(const orc_camera* c, int64_t n, const float* means, const float* scales,
                 const float* quats, uint8_t* flags, int32_t* radius, int32_t* rect,
                 float* depth_key, double* mean2d, double* conic, double* cov2d)
{
    for (int64_t g = 0; g < n; ++g) {
        decision d = decide(c, means + 3 * g, scales + 3 * g, quats + 4 * g);
        flags[g] = (uint8_t)((d.visible ? 1 : 0) | (d.visible && d.degenerate ? 2 : 0));
        radius[g] = d.visible ? d.radius : 0;
        rect[4 * g + 0] = d.visible ? d.x0 : 0;
        rect[4 * g + 1] = d.visible ? d.y0 : 0;
        rect[4 * g + 2] = d.visible ? d.x1 : 0;
        rect[4 * g + 3] = d.visible ? d.y1 : 0;
        depth_key[g] = d.visible ? d.depth_key : 0.0f;
        double m[3], s[3], q[4];
        for (int i = 0; i < 3; ++i) { m[i] = means[3 * g + i]; s[i] = scales[3 * g + i]; }
        for (int i = 0; i < 4; ++i) q[i] = quats[4 * g + i];
        double qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
        double tz = (double)c->R[6] * m[0] + (double)c->R[7] * m[1] + (double)c->R[8] * m[2] + (double)c->t[2];
        if (d.visible && qq > 0.0 && tz > 0.0) {
            project_d(c, m, s, q, mean2d + 2 * g, conic + 3 * g, cov2d ? cov2d + 3 * g : 0);
        } else {
            mean2d[2 * g] = mean2d[2 * g + 1] = 0.0;
            for (int i = 0; i < 3; ++i) { conic[3 * g + i] = 0.0; if (cov2d) cov2d[3 * g + i] = 0.0; }
        }
    }
}

/* Complex-step Jacobian of (u, v, a, b, c) with respect to (m0..2, s0..2, q0..3):
 * jac[g][5][10], row-major.  d f / d x = Im f(x + i h) / h with h = 1e-30. */
void orc_project_jacobian(const orc_camera* c, int64_t n, const double* means, const double* scales,
                          const double* quats, double* jac)
{
    const double h = 1e-30;
    for (int64_t g = 0; g < n; ++g) {
        for (int p = 0; p < 10; ++p) {
            cplx m[3], s[3], q[4], uv[2], cn[3];
            for (int i = 0; i < 3; ++i) { m[i] = means[3 * g + i]; s[i] = scales[3 * g + i]; }
            for (int i = 0; i < 4; ++i) q[i] = quats[4 * g + i];
            if (p < 3) m[p] += I * h;
            else if (p < 6) s[p - 3] += I * h;
            else q[p - 6] += I * h;
            project_c(c, m, s, q, uv, cn, 0);
            double* J = jac + (size_t)g * 50;
            J[0 * 10 + p] = cimag(uv[0]) / h;
            J[1 * 10 + p] = cimag(uv[1]) / h;
            J[2 * 10 + p] = cimag(cn[0]) / h;
            J[3 * 10 + p] = cimag(cn[1]) / h;
            J[4 * 10 + p] = cimag(cn[2]) / h;
        }
    }
}

/* ======================================================================================
 * 3. Binning and depth order: one instance per (visible Gaussian, tile in its rect),
 *    ordered by (tile id = ty*GX + tx, float bits of the depth key, Gaussian id).
 * ==================================================================================== */

typedef struct { uint32_t tile, depth_bits, gid; } inst_key;

static int inst_cmp(const void* pa, const void* pb)
{
    const inst_key* a = (const inst_key*)pa;
    const inst_key* b = (const inst_key*)pb;
    if (a->tile != b->tile) return a->tile < b->tile ? -1 : 1;
    if (a->depth_bits != b->depth_bits) return a->depth_bits < b->depth_bits ? -1 : 1;
    if (a->gid != b->gid) return a->gid < b->gid ? -1 : 1;
    return 0;
}

int64_t orc_count_instances(const orc_camera* c, int64_t n, const uint8_t* flags, const int32_t* rect)
{
    (void)c;
    int64_t total = 0;
    for (int64_t g = 0; g < n; ++g)
        if (flags[g] & 1)
            total += (int64_t)(rect[4 * g + 2] - rect[4 * g + 0]) * (rect[4 * g + 3] - rect[4 * g + 1]);
    return total;
}

/* Fills gauss_ids[I] and tile_ranges[num_tiles][2] = [start, end) with start = number of
 * instances in earlier tiles (so empty tiles have start == end == that prefix). Returns I. */
int64_t orc_bin(const orc_camera* c, int64_t n, const uint8_t* flags, const int32_t* rect,
                const float* depth_key, uint32_t* gauss_ids, uint32_t* tile_ranges)
{
    int32_t GX = grid_x(c), GY = grid_y(c);
    int64_t total = orc_count_instances(c, n, flags, rect);
    inst_key* keys = (inst_key*)malloc(sizeof(inst_key) * (size_t)(total > 0 ? total : 1));
    int64_t k = 0;
    for (int64_t g = 0; g < n; ++g) {
        if (!(flags[g] & 1)) continue;
        uint32_t bits;
        memcpy(&bits, &depth_key[g], 4);
        for (int32_t ty = rect[4 * g + 1]; ty < rect[4 * g + 3]; ++ty)
            for (int32_t tx = rect[4 * g + 0]; tx < rect[4 * g + 2]; ++tx) {
                keys[k].tile = (uint32_t)(ty * GX + tx);
                keys[k].depth_bits = bits;
                keys[k].gid = (uint32_t)g;
                ++k;
            }
    }
    qsort(keys, (size_t)total, sizeof(inst_key), inst_cmp);
    /* ranges as prefix sums: [number of instances in earlier tiles, ... + this tile's count) */
    for (int64_t t = 0; t < (int64_t)GX * GY; ++t) { tile_ranges[2 * t] = 0; tile_ranges[2 * t + 1] = 0; }
    for (int64_t i = 0; i < total; ++i) {
        gauss_ids[i] = keys[i].gid;
        tile_ranges[2 * keys[i].tile + 1] += 1; /* count */
    }
    uint32_t run = 0;
    for (int64_t t = 0; t < (int64_t)GX * GY; ++t) {
        uint32_t cnt = tile_ranges[2 * t + 1];
        tile_ranges[2 * t] = run;
        run += cnt;
        tile_ranges[2 * t + 1] = run;
    }
    free(keys);
    return total;
}

/* ======================================================================================
 * 4. Blending (Eq. 3 with the weights e_i of Eq. 7; Algorithm 1 for the sparse mode).
 *    For each requested pixel (x, y): walk its tile's ordered list front to back.
 *      power = -1/2 (a dx^2 + c dy^2) - b dx dy,  d = mean2d - pixel;  skip if power > 0
 *      alpha = min(0.99, o exp(power));  skip if alpha < 1/255
 *      test_T = T (1 - alpha);  stop (without this Gaussian) if test_T < 1e-4
 *      e = alpha T;  accumulate;  T = test_T
 *    Modes:  0 sparse (Algorithm 1): W_lev[idx_k] += w_k e over the K pairs of each level
 *            1 dense L: W_lev[l] += wd[g][lev][l] e for all l (zeros included)
 *            2 dense D (Eq. 6): F_lev[d] += fd[g][lev][d] e for all d
 *    out[lev][p][ch] (ch < L for modes 0/1, < D for mode 2).
 *    margin[p] = smallest relative distance of a decision quantity (alpha vs 1/255,
 *    test_T vs 1e-4) from its threshold; tiny margins mark knife-edge pixels.
 *    n_eval[p] (optional) = list entries examined, up to and including the one that stops
 *    the walk (the count of evaluations Algorithm 1 makes at this pixel).
 * ==================================================================================== */

void orc_blend(const orc_camera* c, int64_t npix, const int32_t* px, const int32_t* py,
               const double* mean2d, const double* conic, const float* opacity,
               const uint32_t* gauss_ids, const uint32_t* tile_ranges,
               int32_t mode, int32_t levels, int32_t K, int32_t C,
               const uint8_t* idx, const float* w, const double* dense,
               double* out, double* final_T, int32_t* n_last, int32_t* n_contrib, double* margin,
               int32_t* n_eval)
{
    int32_t GX = grid_x(c);
    for (int64_t p = 0; p < npix; ++p) {
        int32_t x = px[p], y = py[p];
        for (int32_t l = 0; l < levels; ++l)
            for (int32_t ch = 0; ch < C; ++ch) out[((size_t)l * npix + p) * C + ch] = 0.0;
        int32_t tile = (y / c->tile_h) * GX + (x / c->tile_w);
        uint32_t beg = tile_ranges[2 * tile], end = tile_ranges[2 * tile + 1];
        double T = 1.0, mg = INFINITY;
        int32_t last = 0, cnt = 0, ev = 0;
        for (uint32_t j = beg; j < end; ++j) {
            uint32_t g = gauss_ids[j];
            ++ev;
            double dx = mean2d[2 * g] - (double)x, dy = mean2d[2 * g + 1] - (double)y;
            double a = conic[3 * g], b = conic[3 * g + 1], cc = conic[3 * g + 2];
            double power = -0.5 * (a * dx * dx + cc * dy * dy) - b * dx * dy;
            if (power > 0.0) continue;
            double alpha = fmin(ORC_ALPHA_MAX, (double)opacity[g] * exp(power));
            double m1 = fabs(alpha - ORC_ALPHA_MIN) / ORC_ALPHA_MIN;
            if (m1 < mg) mg = m1;
            if (alpha < ORC_ALPHA_MIN) continue;
            double test_T = T * (1.0 - alpha);
            double m2 = fabs(test_T - ORC_T_MIN) / ORC_T_MIN;
            if (m2 < mg) mg = m2;
            if (test_T < ORC_T_MIN) break;
            double e = alpha * T;
            for (int32_t l = 0; l < levels; ++l) {
                double* o = out + ((size_t)l * npix + p) * C;
                if (mode == 0) {
                    for (int32_t k = 0; k < K; ++k) {
                        size_t q = ((size_t)g * levels + l) * K + k;
                        o[idx[q]] += (double)w[q] * e;
                    }
                } else {
                    const double* f = dense + ((size_t)g * levels + l) * C;
                    for (int32_t ch = 0; ch < C; ++ch) o[ch] += f[ch] * e;
                }
            }
            T = test_T;
            last = (int32_t)(j - beg + 1);
            ++cnt;
        }
        final_T[p] = T;
        n_last[p] = last;
        if (n_contrib) n_contrib[p] = cnt;
        if (margin) margin[p] = mg;
        if (n_eval) n_eval[p] = ev;
    }
}

/* ======================================================================================
 * 5. Decode (Eq. 7): F_lev = W_lev S_lev, plain triple loop.
 *    W [levels][npix][L], S [levels][L][D] (float), F [levels][npix][D].
 * ==================================================================================== */

void orc_decode(int32_t levels, int64_t npix, int32_t L, int32_t D, const double* W,
                const float* S, double* F)
{
    for (int32_t l = 0; l < levels; ++l)
        for (int64_t p = 0; p < npix; ++p) {
            const double* wp = W + ((size_t)l * npix + p) * L;
            double* fp = F + ((size_t)l * npix + p) * D;
            for (int32_t d = 0; d < D; ++d) {
                double acc = 0.0;
                for (int32_t j = 0; j < L; ++j) acc += wp[j] * (double)S[((size_t)l * L + j) * D + d];
                fp[d] = acc;
            }
        }
}

/* ======================================================================================
 * 6. Relevancy (Sec. 3.2, computed "following LERF"): for each pixel feature F and each
 *    query (one positive t_p, n_neg canonical negatives t_n):
 *       cos(F, t) = <F, t> / (|F| |t|)   (0 when |F| < 1e-12)
 *       rel = min_i  exp(tau cos_p) / (exp(tau cos_p) + exp(tau cos_ni))
 *    F [levels][npix][D], text [Q][1+n_neg][D] (float), rel [Q][levels][npix].
 * ==================================================================================== */

void orc_relevancy(int32_t levels, int64_t npix, int32_t D, const double* F, int32_t Q,
                   int32_t n_neg, const float* text, double tau, double* rel)
{
    for (int32_t l = 0; l < levels; ++l)
        for (int64_t p = 0; p < npix; ++p) {
            const double* f = F + ((size_t)l * npix + p) * D;
            double nf = 0.0;
            for (int32_t d = 0; d < D; ++d) nf += f[d] * f[d];
            nf = sqrt(nf);
            for (int32_t q = 0; q < Q; ++q) {
                double cosv[64];
                for (int32_t k = 0; k <= n_neg; ++k) {
                    const float* t = text + ((size_t)q * (1 + n_neg) + k) * D;
                    double dot = 0.0, nt = 0.0;
                    for (int32_t d = 0; d < D; ++d) { dot += f[d] * (double)t[d]; nt += (double)t[d] * (double)t[d]; }
                    cosv[k] = (nf < 1e-12) ? 0.0 : dot / (nf * sqrt(nt));
                }
                double best = INFINITY;
                for (int32_t k = 1; k <= n_neg; ++k) {
                    double zp = tau * cosv[0], zn = tau * cosv[k];
                    double mx = zp > zn ? zp : zn;
                    double ep = exp(zp - mx), en = exp(zn - mx);
                    double s = ep / (ep + en);
                    if (s < best) best = s;
                }
                rel[((size_t)q * levels + l) * npix + p] = best;
            }
        }
}

/* ======================================================================================
 * 7. Gradient of the blend.  Given G = dLoss/dW [levels][P][L] for every pixel of the
 *    image, accumulate per Gaussian:
 *      dw[g][lev][k]   = sum_p G_lev[idx_k](p) e_g(p)
 *      dalpha_g(p)     = sum_lev,l G_lev,l dW_lev,l/dalpha_g with
 *                        dW_l/dalpha_i = w_il T_i - sum_{j>i} w_jl alpha_j T_j / (1 - alpha_i)
 *                        (literal derivative of W_l = sum_i w_il alpha_i prod_{m<i}(1-alpha_m))
 *      alpha = o exp(power) (unclamped): do += dalpha exp(power), dpower = dalpha alpha
 *      du += dpower * dpower/du, etc. (power as in the blend, d = (u - x, v - y))
 *    Outputs per Gaussian: dw [N][levels][K], dopac [N], dmean2d [N][2], dconic [N][3].
 *    The contributor set and order are those of the forward (same decisions).
 * ==================================================================================== */

void orc_blend_backward(const orc_camera* c, int64_t n, const double* mean2d, const double* conic,
                        const float* opacity, const uint32_t* gauss_ids, const uint32_t* tile_ranges,
                        int32_t levels, int32_t K, int32_t L, const uint8_t* idx, const float* w,
                        const double* G, double* dw, double* dopac, double* dmean2d, double* dconic)
{
    int32_t GX = grid_x(c);
    int64_t P = (int64_t)c->width * c->height;
    memset(dw, 0, sizeof(double) * (size_t)n * levels * K);
    memset(dopac, 0, sizeof(double) * (size_t)n);
    memset(dmean2d, 0, sizeof(double) * (size_t)n * 2);
    memset(dconic, 0, sizeof(double) * (size_t)n * 3);
    /* per-pixel contributor record */
    typedef struct { uint32_t g; double alpha, T, ex, dx, dy; int clamped; } contrib;
    size_t cap = 1024;
    contrib* cs = (contrib*)malloc(sizeof(contrib) * cap);
    double* gsum = (double*)malloc(sizeof(double) * cap);
    for (int32_t y = 0; y < c->height; ++y)
        for (int32_t x = 0; x < c->width; ++x) {
            int64_t p = (int64_t)y * c->width + x;
            int32_t tile = (y / c->tile_h) * GX + (x / c->tile_w);
            uint32_t beg = tile_ranges[2 * tile], end = tile_ranges[2 * tile + 1];
            double T = 1.0;
            size_t nc = 0;
            for (uint32_t j = beg; j < end; ++j) {
                uint32_t g = gauss_ids[j];
                double dx = mean2d[2 * g] - (double)x, dy = mean2d[2 * g + 1] - (double)y;
                double a = conic[3 * g], b = conic[3 * g + 1], cc = conic[3 * g + 2];
                double power = -0.5 * (a * dx * dx + cc * dy * dy) - b * dx * dy;
                if (power > 0.0) continue;
                double ex = exp(power);
                double raw = (double)opacity[g] * ex;
                double alpha = fmin(ORC_ALPHA_MAX, raw);
                if (alpha < ORC_ALPHA_MIN) continue;
                double test_T = T * (1.0 - alpha);
                if (test_T < ORC_T_MIN) break;
                if (nc == cap) {
                    cap *= 2;
                    cs = (contrib*)realloc(cs, sizeof(contrib) * cap);
                    gsum = (double*)realloc(gsum, sizeof(double) * cap);
                }
                cs[nc].g = g; cs[nc].alpha = alpha; cs[nc].T = T; cs[nc].ex = ex;
                cs[nc].dx = dx; cs[nc].dy = dy; cs[nc].clamped = raw > ORC_ALPHA_MAX;
                ++nc;
                T = test_T;
            }
            /* g_i = sum_lev sum_k G_lev[idx_ik] w_ik  (dLoss/de_i) */
            for (size_t i = 0; i < nc; ++i) {
                uint32_t g = cs[i].g;
                double e = cs[i].alpha * cs[i].T, s = 0.0;
                for (int32_t l = 0; l < levels; ++l)
                    for (int32_t k = 0; k < K; ++k) {
                        size_t q = ((size_t)g * levels + l) * K + k;
                        double gl = G[((size_t)l * P + p) * L + idx[q]];
                        dw[q] += gl * e;
                        s += gl * (double)w[q];
                    }
                gsum[i] = s;
            }
            for (size_t i = 0; i < nc; ++i) {
                double later = 0.0;
                for (size_t j = i + 1; j < nc; ++j) later += gsum[j] * cs[j].alpha * cs[j].T;
                double dalpha = gsum[i] * cs[i].T - later / (1.0 - cs[i].alpha);
                if (cs[i].clamped) continue;
                uint32_t g = cs[i].g;
                double a = conic[3 * g], b = conic[3 * g + 1], cc = conic[3 * g + 2];
                double dx = cs[i].dx, dy = cs[i].dy;
                dopac[g] += dalpha * cs[i].ex;
                double dpow = dalpha * cs[i].alpha;
                dmean2d[2 * g] += dpow * (-(a * dx + b * dy));
                dmean2d[2 * g + 1] += dpow * (-(b * dx + cc * dy));
                dconic[3 * g] += dpow * (-0.5 * dx * dx);
                dconic[3 * g + 1] += dpow * (-dx * dy);
                dconic[3 * g + 2] += dpow * (-0.5 * dy * dy);
            }
        }
    free(cs);
    free(gsum);
}

/* ======================================================================================
 * 8. FD support: the L1 loss of Sec. 3.3's feature rendering against a target, with
 *    FP64 parameters, a FIXED tile list (the binning of the base parameters) and a
 *    restricted set of tiles.  Returns sum_p,d |F - T_gt| over pixels of the tiles with
 *    tile_mask != 0 (divide by P*D outside), optionally each pixel's own sum (so that a
 *    central difference can cancel untouched pixels exactly), and a 64-bit signature of every discrete
 *    decision taken (contributor set, clamp flags, termination, L1 signs) so that a
 *    finite difference that crosses a branch can be recognised and left out.
 * ==================================================================================== */

static uint64_t mix64(uint64_t h, uint64_t v)
{
    h ^= v + 0x9e3779b97f4a7c15ULL + (h << 6) + (h >> 2);
    return h;
}

double orc_l1_loss_tiles(const orc_camera* c, int64_t n, const double* means, const double* scales,
                         const double* quats, const double* opacity, const uint32_t* gauss_ids,
                         const uint32_t* tile_ranges, const uint8_t* tile_mask, int32_t levels,
                         int32_t K, int32_t L, int32_t D, const uint8_t* idx, const double* w,
                         const float* S, const float* target, double* per_pixel,
                         uint64_t* signature)
{
    int32_t GX = grid_x(c), GY = grid_y(c);
    int64_t P = (int64_t)c->width * c->height;
    double* uv = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    double* cn = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    for (int64_t g = 0; g < n; ++g)
        project_d(c, means + 3 * g, scales + 3 * g, quats + 4 * g, uv + 2 * g, cn + 3 * g, 0);
    double* W = (double*)malloc(sizeof(double) * (size_t)levels * L);
    double loss = 0.0;
    uint64_t sig = 1469598103934665603ULL;
    for (int32_t ty = 0; ty < GY; ++ty)
        for (int32_t tx = 0; tx < GX; ++tx) {
            int32_t tile = ty * GX + tx;
            if (!tile_mask[tile]) continue;
            uint32_t beg = tile_ranges[2 * tile], end = tile_ranges[2 * tile + 1];
            for (int32_t y = ty * c->tile_h; y < (ty + 1) * c->tile_h && y < c->height; ++y)
                for (int32_t x = tx * c->tile_w; x < (tx + 1) * c->tile_w && x < c->width; ++x) {
                    memset(W, 0, sizeof(double) * (size_t)levels * L);
                    double T = 1.0;
                    for (uint32_t j = beg; j < end; ++j) {
                        uint32_t g = gauss_ids[j];
                        double dx = uv[2 * g] - x, dy = uv[2 * g + 1] - y;
                        double power = -0.5 * (cn[3 * g] * dx * dx + cn[3 * g + 2] * dy * dy) - cn[3 * g + 1] * dx * dy;
                        if (power > 0.0) continue;
                        double raw = opacity[g] * exp(power);
                        double alpha = fmin(ORC_ALPHA_MAX, raw);
                        if (alpha < ORC_ALPHA_MIN) continue;
                        double test_T = T * (1.0 - alpha);
                        if (test_T < ORC_T_MIN) { sig = mix64(sig, 0xDEADull + j); break; }
                        sig = mix64(sig, ((uint64_t)j << 1) | (raw > ORC_ALPHA_MAX ? 1u : 0u));
                        double e = alpha * T;
                        for (int32_t l = 0; l < levels; ++l)
                            for (int32_t k = 0; k < K; ++k) {
                                size_t q = ((size_t)g * levels + l) * K + k;
                                W[l * L + idx[q]] += w[q] * e;
                            }
                        T = test_T;
                    }
                    int64_t p = (int64_t)y * c->width + x;
                    double lp = 0.0;
                    for (int32_t l = 0; l < levels; ++l)
                        for (int32_t d = 0; d < D; ++d) {
                            double f = 0.0;
                            for (int32_t j = 0; j < L; ++j) f += W[l * L + j] * (double)S[((size_t)l * L + j) * D + d];
                            double r = f - (double)target[((size_t)l * P + p) * D + d];
                            lp += fabs(r);
                            sig = mix64(sig, r > 0.0 ? 3u : (r < 0.0 ? 5u : 7u));
                        }
                    if (per_pixel) per_pixel[p] = lp;
                    loss += lp;
                }
        }
    free(uv);
    free(cn);
    free(W);
    if (signature) *signature = sig;
    return loss;
}

/* FP64 projection with double inputs (for finite-difference checks of the Jacobian). */
void orc_project64(const orc_camera* c, int64_t n, const double* means, const double* scales,
                   const double* quats, double* mean2d, double* conic)
{
    for (int64_t g = 0; g < n; ++g)
        project_d(c, means + 3 * g, scales + 3 * g, quats + 4 * g, mean2d + 2 * g, conic + 3 * g, 0);
}

/* ======================================================================================
 * 8. Post-processing of the relevancy maps M (paper appendix, "Evaluation Details").
 *    Mean filter ("average pooling", Avg(M)): out(x, y) is the mean of M over the pixels of
 *    the k x k window centred on (x, y) that lie inside the image (k odd; the paper gives no
 *    window size or border rule).
 *    mode 0 (LERF): S = Avg(M) per level; the selected level is the one whose S has the
 *      highest value (lowest level on a tie); the localisation point is the first pixel in
 *      row-major order where that level's S is maximal; the segmentation mask is
 *      (S - min S) / (max S - min S) > thr on that level (0 everywhere when max = min).
 *    mode 1 (3D-OVS, Mip-NeRF360): S = 0.5 (M + Avg(M)); each level's mask as above; the
 *      selected level has the highest mean of S over its own mask (an empty mask counts as
 *      -infinity; lowest level on a tie); point and mask as in mode 0.
 *    rel [levels][H*W] one query; smoothed [levels][H*W]; point = (x, y); mask [H*W].
 * ==================================================================================== */

void orc_mean_filter(int32_t H, int32_t W, int32_t k, const double* in, double* out)
{
    const int32_t r = (k - 1) / 2;
    for (int32_t y = 0; y < H; ++y)
        for (int32_t x = 0; x < W; ++x) {
            const int32_t y0 = y - r < 0 ? 0 : y - r, y1 = y + r > H - 1 ? H - 1 : y + r;
            const int32_t x0 = x - r < 0 ? 0 : x - r, x1 = x + r > W - 1 ? W - 1 : x + r;
            double sum = 0.0;
            for (int32_t yy = y0; yy <= y1; ++yy)
                for (int32_t xx = x0; xx <= x1; ++xx) sum += in[(size_t)yy * W + xx];
            out[(size_t)y * W + x] = sum / (double)((y1 - y0 + 1) * (x1 - x0 + 1));
        }
}

static void normalised_mask(int64_t P, const double* s, double thr, uint8_t* mask)
{
    double mx = -INFINITY, mn = INFINITY;
    for (int64_t p = 0; p < P; ++p) {
        if (s[p] > mx) mx = s[p];
        if (s[p] < mn) mn = s[p];
    }
    for (int64_t p = 0; p < P; ++p) {
        const double nrm = mx > mn ? (s[p] - mn) / (mx - mn) : 0.0;
        mask[p] = nrm > thr ? 1 : 0;
    }
}

void orc_postprocess(int32_t levels, int32_t H, int32_t W, const double* rel, int32_t k, int32_t mode,
                     double thr, double* smoothed, int32_t* point, int32_t* level, double* score,
                     uint8_t* mask)
{
    const int64_t P = (int64_t)H * W;
    for (int32_t l = 0; l < levels; ++l) {
        double* s = smoothed + (size_t)l * P;
        orc_mean_filter(H, W, k, rel + (size_t)l * P, s);
        if (mode == 1)
            for (int64_t p = 0; p < P; ++p) s[p] = 0.5 * (rel[(size_t)l * P + p] + s[p]);
    }
    int32_t sel = 0;
    double best = -INFINITY;
    for (int32_t l = 0; l < levels; ++l) {
        const double* s = smoothed + (size_t)l * P;
        double crit;
        if (mode == 0) {
            crit = -INFINITY;
            for (int64_t p = 0; p < P; ++p)
                if (s[p] > crit) crit = s[p];
        } else {
            normalised_mask(P, s, thr, mask);
            double sum = 0.0;
            int64_t cnt = 0;
            for (int64_t p = 0; p < P; ++p)
                if (mask[p]) { sum += s[p]; ++cnt; }
            crit = cnt > 0 ? sum / (double)cnt : -INFINITY;
        }
        if (l == 0 || crit > best) { best = crit; sel = l; }
    }
    const double* s = smoothed + (size_t)sel * P;
    int64_t arg = 0;
    for (int64_t p = 1; p < P; ++p)
        if (s[p] > s[arg]) arg = p;
    point[0] = (int32_t)(arg % W);
    point[1] = (int32_t)(arg / W);
    *level = sel;
    *score = s[arg];
    normalised_mask(P, s, thr, mask);
}
