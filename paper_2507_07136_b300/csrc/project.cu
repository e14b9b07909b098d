// project.cu -- EWA projection of 3D Gaussians (Sec. 3.1, Eq. 1-2), one thread per Gaussian.
//
// Two evaluations of the same geometry:
//  * The decision path decides visibility, the screen radius, the tile rectangle and the
//    depth key.  It is a fixed sequence of correctly rounded float32 operations (explicit
//    __f*_rn intrinsics, so nothing is contracted or reordered), which makes those integers
//    reproducible bit for bit by any IEEE implementation of the same sequence.  The 2D
//    covariance is formed as N N^T with N = J W R diag(s) (2x3): its determinant is the
//    squared norm of the cross product of N's rows, which has no cancellation.  When the
//    undilated covariance is near-degenerate (tr^2 >= 1e6 det) the covariance part and the
//    depth key are re-evaluated in FP64.
//  * The value path computes the 2D mean and the conic that the blend uses, in double-float
//    arithmetic.  A float32 2D mean at u ~ 1000 px carries ~1e-4 px of error from the
//    camera transform alone, which moves alpha by ~1e-4 relative at the footprint edge; the
//    double-float mean is stored as a (hi, lo) pair so the blend can form u - x exactly.  The
//    same path produces the conic's principal frame (stiff axis as a float pair, eigenvalues)
//    in which the blend evaluates the Gaussian without cancellation.
#include "device.cuh"
#include "project.cuh"

namespace lsv2 {
namespace {

#define FADD __fadd_rn
#define FSUB __fsub_rn
#define FMUL __fmul_rn
#define FDIV __fdiv_rn
#define FSQRT __fsqrt_rn
#define DADD __dadd_rn
#define DSUB __dsub_rn
#define DMUL __dmul_rn
#define DDIV __ddiv_rn
#define DSQRT __dsqrt_rn

struct ProjectArgs {
    lsv2_camera cam[kMaxProjectViews];   // one camera per view (blockIdx.y)
    int64_t n;
    const float* means;
    const float* scales;
    const float* quats;
    const float* opacity;
    lsv2_proj out;
    int32_t* status;
};

__device__ int32_t clamp_floor(float f, int32_t lo, int32_t hi)
{
    if (!(f >= (float)lo)) return lo;
    if (f > (float)hi) return hi;
    return (int32_t)f;
}

// FP64 covariance/radius decision for near-degenerate Gaussians (same steps as the float32
// path, from the exactly widened float inputs).
__device__ int32_t degenerate_radius(const lsv2_camera& c, const float m[3], const float s[3],
                                     const float q[4], float* depth_key)
{
    double t[3];
    for (int i = 0; i < 3; ++i)
        t[i] = DADD(DADD(DADD(DMUL((double)c.R[3 * i], (double)m[0]), DMUL((double)c.R[3 * i + 1], (double)m[1])),
                         DMUL((double)c.R[3 * i + 2], (double)m[2])),
                    (double)c.t[i]);
    double n2 = DADD(DADD(DADD(DMUL((double)q[0], (double)q[0]), DMUL((double)q[1], (double)q[1])),
                          DMUL((double)q[2], (double)q[2])),
                     DMUL((double)q[3], (double)q[3]));
    double inv = DDIV(1.0, DSQRT(n2));
    double w = DMUL((double)q[0], inv), x = DMUL((double)q[1], inv), y = DMUL((double)q[2], inv),
           z = DMUL((double)q[3], inv);
    double R[9];
    R[0] = DSUB(1.0, DMUL(2.0, DADD(DMUL(y, y), DMUL(z, z))));
    R[1] = DMUL(2.0, DSUB(DMUL(x, y), DMUL(w, z)));
    R[2] = DMUL(2.0, DADD(DMUL(x, z), DMUL(w, y)));
    R[3] = DMUL(2.0, DADD(DMUL(x, y), DMUL(w, z)));
    R[4] = DSUB(1.0, DMUL(2.0, DADD(DMUL(x, x), DMUL(z, z))));
    R[5] = DMUL(2.0, DSUB(DMUL(y, z), DMUL(w, x)));
    R[6] = DMUL(2.0, DSUB(DMUL(x, z), DMUL(w, y)));
    R[7] = DMUL(2.0, DADD(DMUL(y, z), DMUL(w, x)));
    R[8] = DSUB(1.0, DMUL(2.0, DADD(DMUL(x, x), DMUL(y, y))));
    double M[9];
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j) M[3 * k + j] = DMUL(R[3 * k + j], (double)s[j]);
    double tanx = DDIV((double)c.width, DMUL(2.0, (double)c.fx));
    double tany = DDIV((double)c.height, DMUL(2.0, (double)c.fy));
    double limx = DMUL((double)kGuard, tanx), limy = DMUL((double)kGuard, tany);
    double txz = DDIV(t[0], t[2]), tyz = DDIV(t[1], t[2]);
    double cxz = fmin(limx, fmax(-limx, txz)), cyz = fmin(limy, fmax(-limy, tyz));
    double J00 = DDIV((double)c.fx, t[2]), J11 = DDIV((double)c.fy, t[2]);
    double J02 = -DDIV(DMUL((double)c.fx, cxz), t[2]);
    double J12 = -DDIV(DMUL((double)c.fy, cyz), t[2]);
    double T[6];
    for (int j = 0; j < 3; ++j) {
        T[j] = DADD(DMUL(J00, (double)c.R[j]), DMUL(J02, (double)c.R[6 + j]));
        T[3 + j] = DADD(DMUL(J11, (double)c.R[3 + j]), DMUL(J12, (double)c.R[6 + j]));
    }
    double N[6];
    for (int a = 0; a < 2; ++a)
        for (int j = 0; j < 3; ++j)
            N[3 * a + j] = DADD(DADD(DMUL(T[3 * a], M[j]), DMUL(T[3 * a + 1], M[3 + j])), DMUL(T[3 * a + 2], M[6 + j]));
    double s00 = DADD(DADD(DMUL(N[0], N[0]), DMUL(N[1], N[1])), DMUL(N[2], N[2]));
    double s11 = DADD(DADD(DMUL(N[3], N[3]), DMUL(N[4], N[4])), DMUL(N[5], N[5]));
    double s01 = DADD(DADD(DMUL(N[0], N[3]), DMUL(N[1], N[4])), DMUL(N[2], N[5]));
    double d = (double)kDilation;
    double mid = DMUL(0.5, DADD(DADD(s00, d), DADD(s11, d)));
    double hd = DMUL(0.5, DSUB(s00, s11));
    double disc = fmax((double)kDiscFloor, DADD(DMUL(hd, hd), DMUL(s01, s01)));
    double lam = DADD(mid, DSQRT(disc));
    double rf = ceil(DMUL(3.0, DSQRT(lam)));
    if (!(rf < (double)kRadiusCap)) rf = (double)kRadiusCap;
    *depth_key = __double2float_rn(t[2]);
    return (int32_t)rf;
}

__global__ void __launch_bounds__(256, 4) project_kernel(ProjectArgs a)   // 4 blocks per SM: latency-bound
{
    const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= a.n) return;
    const lsv2_camera& c = a.cam[blockIdx.y];
    const int64_t g = gi;                                 // Gaussian (inputs)
    const int64_t o = (int64_t)blockIdx.y * a.n + gi;     // output slot of this view
    float m[3] = {a.means[3 * g], a.means[3 * g + 1], a.means[3 * g + 2]};
    float s[3] = {a.scales[3 * g], a.scales[3 * g + 1], a.scales[3 * g + 2]};
    float4 q4 = reinterpret_cast<const float4*>(a.quats)[g];
    float q[4] = {q4.x, q4.y, q4.z, q4.w};
    float opac = a.opacity[g];

    // ---- decision path (float32, fixed order) ----
    float t0 = FADD(FADD(FADD(FMUL(c.R[0], m[0]), FMUL(c.R[1], m[1])), FMUL(c.R[2], m[2])), c.t[0]);
    float t1 = FADD(FADD(FADD(FMUL(c.R[3], m[0]), FMUL(c.R[4], m[1])), FMUL(c.R[5], m[2])), c.t[1]);
    float t2 = FADD(FADD(FADD(FMUL(c.R[6], m[0]), FMUL(c.R[7], m[1])), FMUL(c.R[8], m[2])), c.t[2]);
    float n2 = FADD(FADD(FADD(FMUL(q[0], q[0]), FMUL(q[1], q[1])), FMUL(q[2], q[2])), FMUL(q[3], q[3]));
    bool visible = (t2 > c.near_z) && (n2 > 0.0f);
    int32_t radius = 0, x0 = 0, y0 = 0, x1 = 0, y1 = 0;
    float depth_key = 0.0f;
    bool degenerate = false;
    if (visible) {
        float inv = FDIV(1.0f, FSQRT(n2));
        float w = FMUL(q[0], inv), x = FMUL(q[1], inv), y = FMUL(q[2], inv), z = FMUL(q[3], inv);
        float R[9];
        R[0] = FSUB(1.0f, FMUL(2.0f, FADD(FMUL(y, y), FMUL(z, z))));
        R[1] = FMUL(2.0f, FSUB(FMUL(x, y), FMUL(w, z)));
        R[2] = FMUL(2.0f, FADD(FMUL(x, z), FMUL(w, y)));
        R[3] = FMUL(2.0f, FADD(FMUL(x, y), FMUL(w, z)));
        R[4] = FSUB(1.0f, FMUL(2.0f, FADD(FMUL(x, x), FMUL(z, z))));
        R[5] = FMUL(2.0f, FSUB(FMUL(y, z), FMUL(w, x)));
        R[6] = FMUL(2.0f, FSUB(FMUL(x, z), FMUL(w, y)));
        R[7] = FMUL(2.0f, FADD(FMUL(y, z), FMUL(w, x)));
        R[8] = FSUB(1.0f, FMUL(2.0f, FADD(FMUL(x, x), FMUL(y, y))));
        float M[9];
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j) M[3 * k + j] = FMUL(R[3 * k + j], s[j]);
        float tanx = FDIV((float)c.width, FMUL(2.0f, c.fx));
        float tany = FDIV((float)c.height, FMUL(2.0f, c.fy));
        float limx = FMUL(kGuard, tanx), limy = FMUL(kGuard, tany);
        float txz = FDIV(t0, t2), tyz = FDIV(t1, t2);
        float cxz = fminf(limx, fmaxf(-limx, txz)), cyz = fminf(limy, fmaxf(-limy, tyz));
        float J00 = FDIV(c.fx, t2), J11 = FDIV(c.fy, t2);
        float J02 = -FDIV(FMUL(c.fx, cxz), t2), J12 = -FDIV(FMUL(c.fy, cyz), t2);
        float T[6];
        for (int j = 0; j < 3; ++j) {
            T[j] = FADD(FMUL(J00, c.R[j]), FMUL(J02, c.R[6 + j]));
            T[3 + j] = FADD(FMUL(J11, c.R[3 + j]), FMUL(J12, c.R[6 + j]));
        }
        float N[6];
        for (int r = 0; r < 2; ++r)
            for (int j = 0; j < 3; ++j)
                N[3 * r + j] = FADD(FADD(FMUL(T[3 * r], M[j]), FMUL(T[3 * r + 1], M[3 + j])), FMUL(T[3 * r + 2], M[6 + j]));
        float s00 = FADD(FADD(FMUL(N[0], N[0]), FMUL(N[1], N[1])), FMUL(N[2], N[2]));
        float s11 = FADD(FADD(FMUL(N[3], N[3]), FMUL(N[4], N[4])), FMUL(N[5], N[5]));
        float s01 = FADD(FADD(FMUL(N[0], N[3]), FMUL(N[1], N[4])), FMUL(N[2], N[5]));
        float k0 = FSUB(FMUL(N[1], N[5]), FMUL(N[2], N[4]));
        float k1 = FSUB(FMUL(N[2], N[3]), FMUL(N[0], N[5]));
        float k2 = FSUB(FMUL(N[0], N[4]), FMUL(N[1], N[3]));
        float det0 = FADD(FADD(FMUL(k0, k0), FMUL(k1, k1)), FMUL(k2, k2));
        float tr = FADD(s00, s11);
        degenerate = !(FMUL(det0, kDegenerateCond) > FMUL(tr, tr));
        if (!degenerate) {
            float mid = FMUL(0.5f, FADD(FADD(s00, kDilation), FADD(s11, kDilation)));
            float hd = FMUL(0.5f, FSUB(s00, s11));
            float disc = fmaxf(kDiscFloor, FADD(FMUL(hd, hd), FMUL(s01, s01)));
            float lam = FADD(mid, FSQRT(disc));
            float rf = ceilf(FMUL(3.0f, FSQRT(lam)));
            if (!(rf < kRadiusCap)) rf = kRadiusCap;
            radius = (int32_t)rf;
            depth_key = t2;
        } else {
            radius = degenerate_radius(c, m, s, q, &depth_key);
        }
        float u = FADD(FMUL(c.fx, txz), c.cx);
        float v = FADD(FMUL(c.fy, tyz), c.cy);
        float r = (float)radius;
        float tw = (float)c.tile_w, th = (float)c.tile_h;
        int32_t GX = (c.width + c.tile_w - 1) / c.tile_w, GY = (c.height + c.tile_h - 1) / c.tile_h;
        x0 = clamp_floor(floorf(FDIV(FSUB(u, r), tw)), 0, GX);
        x1 = clamp_floor(floorf(FDIV(FADD(FADD(u, r), FSUB(tw, 1.0f)), tw)), 0, GX);
        y0 = clamp_floor(floorf(FDIV(FSUB(v, r), th)), 0, GY);
        y1 = clamp_floor(floorf(FDIV(FADD(FADD(v, r), FSUB(th, 1.0f)), th)), 0, GY);
        visible = (x1 > x0) && (y1 > y0);
    }

    float4 xy = make_float4(0.f, 0.f, 0.f, 0.f), cn = make_float4(0.f, 0.f, 0.f, opac);
    float2 ext = make_float2(-1.0f, -1.0f);
    float4 ax0 = make_float4(0.f, 0.f, 0.f, 0.f), ax1 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (visible) {
        // ---- value path (double-float) ----
        dfloat td[3];
        for (int i = 0; i < 3; ++i) {
            dfloat acc = df_add(two_prod(c.R[3 * i], m[0]), two_prod(c.R[3 * i + 1], m[1]));
            acc = df_add(acc, two_prod(c.R[3 * i + 2], m[2]));
            td[i] = df_add(acc, df(c.t[i]));
        }
        dfloat txz = df_div(td[0], td[2]), tyz = df_div(td[1], td[2]);
        dfloat u = df_add(df_mul_f(txz, c.fx), df(c.cx));
        dfloat v = df_add(df_mul_f(tyz, c.fy), df(c.cy));
        xy = make_float4(u.hi, v.hi, u.lo, v.lo);

        // rotation of the (unnormalised) quaternion: R = Q(q) / |q|^2
        dfloat ww = two_prod(q[0], q[0]), xx = two_prod(q[1], q[1]), yy = two_prod(q[2], q[2]),
               zz = two_prod(q[3], q[3]);
        dfloat xy_ = two_prod(q[1], q[2]), xz = two_prod(q[1], q[3]), yz = two_prod(q[2], q[3]);
        dfloat wx = two_prod(q[0], q[1]), wy = two_prod(q[0], q[2]), wz = two_prod(q[0], q[3]);
        dfloat nq = df_add(df_add(ww, xx), df_add(yy, zz));
        dfloat inv = df_div(df(1.0f), nq);
        dfloat R[9];
        R[0] = df_mul(df_sub(df_add(ww, xx), df_add(yy, zz)), inv);
        R[1] = df_mul(df_mul_f(df_sub(xy_, wz), 2.0f), inv);
        R[2] = df_mul(df_mul_f(df_add(xz, wy), 2.0f), inv);
        R[3] = df_mul(df_mul_f(df_add(xy_, wz), 2.0f), inv);
        R[4] = df_mul(df_sub(df_add(ww, yy), df_add(xx, zz)), inv);
        R[5] = df_mul(df_mul_f(df_sub(yz, wx), 2.0f), inv);
        R[6] = df_mul(df_mul_f(df_sub(xz, wy), 2.0f), inv);
        R[7] = df_mul(df_mul_f(df_add(yz, wx), 2.0f), inv);
        R[8] = df_mul(df_sub(df_add(ww, zz), df_add(xx, yy)), inv);
        dfloat M[9];
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j) M[3 * k + j] = df_mul_f(R[3 * k + j], s[j]);
        float limx = FMUL(kGuard, FDIV((float)c.width, FMUL(2.0f, c.fx)));
        float limy = FMUL(kGuard, FDIV((float)c.height, FMUL(2.0f, c.fy)));
        dfloat cxz = txz.hi > limx ? df(limx) : (txz.hi < -limx ? df(-limx) : txz);
        dfloat cyz = tyz.hi > limy ? df(limy) : (tyz.hi < -limy ? df(-limy) : tyz);
        dfloat J00 = df_div(df(c.fx), td[2]), J11 = df_div(df(c.fy), td[2]);
        dfloat J02 = df_neg(df_div(df_mul_f(cxz, c.fx), td[2]));
        dfloat J12 = df_neg(df_div(df_mul_f(cyz, c.fy), td[2]));
        dfloat T[6];
        for (int j = 0; j < 3; ++j) {
            T[j] = df_add(df_mul_f(J00, c.R[j]), df_mul_f(J02, c.R[6 + j]));
            T[3 + j] = df_add(df_mul_f(J11, c.R[3 + j]), df_mul_f(J12, c.R[6 + j]));
        }
        dfloat N[6];
        for (int r = 0; r < 2; ++r)
            for (int j = 0; j < 3; ++j)
                N[3 * r + j] = df_add(df_add(df_mul(T[3 * r], M[j]), df_mul(T[3 * r + 1], M[3 + j])),
                                      df_mul(T[3 * r + 2], M[6 + j]));
        dfloat s00 = df_add(df_add(df_mul(N[0], N[0]), df_mul(N[1], N[1])), df_mul(N[2], N[2]));
        dfloat s11 = df_add(df_add(df_mul(N[3], N[3]), df_mul(N[4], N[4])), df_mul(N[5], N[5]));
        dfloat s01 = df_add(df_add(df_mul(N[0], N[3]), df_mul(N[1], N[4])), df_mul(N[2], N[5]));
        dfloat k0 = df_sub(df_mul(N[1], N[5]), df_mul(N[2], N[4]));
        dfloat k1 = df_sub(df_mul(N[2], N[3]), df_mul(N[0], N[5]));
        dfloat k2 = df_sub(df_mul(N[0], N[4]), df_mul(N[1], N[3]));
        dfloat det0 = df_add(df_add(df_mul(k0, k0), df_mul(k1, k1)), df_mul(k2, k2));
        // det(Sigma' + d I) = det0 + d tr + d^2   (no cancellation)
        dfloat det = df_add(df_add(det0, df_mul_f(df_add(s00, s11), kDilation)), two_prod(kDilation, kDilation));
        dfloat c00 = df_add(s00, df(kDilation)), c11 = df_add(s11, df(kDilation));
        float ca = df_div(c11, det).hi, cb = -df_div(s01, det).hi, cc = df_div(c00, det).hi;
        cn = make_float4(ca, cb, cc, opac);
        // principal frame: the covariance's long axis is the conic's soft axis
        dfloat hd = df_mul_f(df_sub(c00, c11), 0.5f);
        dfloat r = df_sqrt(df_add(df_mul(hd, hd), df_mul(s01, s01)));
        dfloat lmax = df_add(df_mul_f(df_add(c00, c11), 0.5f), r);
        dfloat lmin = df_div(det, lmax);
        dfloat sx = df(1.0f), sy = df(0.0f);
        if (r.hi > 0.0f) {
            dfloat x = hd.hi >= 0.0f ? df_add(hd, r) : s01;
            dfloat y = hd.hi >= 0.0f ? s01 : df_sub(r, hd);
            dfloat nrm = df_sqrt(df_add(df_mul(x, x), df_mul(y, y)));
            sx = df_div(x, nrm);
            sy = df_div(y, nrm);
        }
        const float q1 = df_div(df(1.0f), lmin).hi, q2 = df_div(df(1.0f), lmax).hi;
        // stiff axis = soft axis rotated by +90 degrees: (-sy, sx)
        ax0 = make_float4(-sy.hi, sx.hi, -0.5f * kLog2e * q1, -0.5f * kLog2e * q2);
        ax1 = make_float4(-sy.lo, sx.lo, __fdiv_rn(lmax.hi, lmin.hi), 0.0f);
        // bounding box of {alpha >= 1/255}: d^T Q d <= 2 ln(255 o); half-widths sqrt(t c00),
        // sqrt(t c11).  Widened by 1e-3 relative so float rounding in the blend can never
        // put a contributing pixel outside it.
        if (opac * 255.0f > 1.0f) {
            float tcut = 2.0f * logf(255.0f * opac) * 1.001f + 1e-3f;
            ext = make_float2(sqrtf(tcut * c00.hi) + 1e-3f, sqrtf(tcut * c11.hi) + 1e-3f);
        }
    }
    reinterpret_cast<float4*>(a.out.xy)[o] = xy;
    reinterpret_cast<float4*>(a.out.conic_o)[o] = cn;
    reinterpret_cast<float2*>(a.out.extent)[o] = ext;
    reinterpret_cast<float4*>(a.out.axes)[2 * o] = ax0;
    reinterpret_cast<float4*>(a.out.axes)[2 * o + 1] = ax1;
    a.out.depth[o] = visible ? depth_key : 0.0f;
    a.out.radius[o] = visible ? radius : 0;
    reinterpret_cast<int4*>(a.out.rect)[o] = visible ? make_int4(x0, y0, x1, y1) : make_int4(0, 0, 0, 0);
    a.out.tiles_touched[o] = visible ? (uint32_t)((x1 - x0) * (y1 - y0)) : 0u;
    a.out.flags[o] = (uint8_t)((visible ? 1 : 0) | (visible && degenerate ? 2 : 0));
}

}  // namespace

cudaError_t launch_project(const lsv2_camera* cams, int V, int64_t n, const float* means, const float* scales,
                           const float* quats, const float* opacity, const lsv2_proj& out, int32_t* status,
                           cudaStream_t stream)
{
    if (n == 0 || V == 0) return cudaSuccess;
    if (V > kMaxProjectViews) return cudaErrorInvalidValue;
    ProjectArgs a{};
    for (int v = 0; v < V; ++v) a.cam[v] = cams[v];
    a.n = n;
    a.means = means;
    a.scales = scales;
    a.quats = quats;
    a.opacity = opacity;
    a.out = out;
    a.status = status;
    const int threads = 256;
    const int64_t blocks = (n + threads - 1) / threads;
    project_kernel<<<dim3((unsigned)blocks, (unsigned)V), threads, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace lsv2
