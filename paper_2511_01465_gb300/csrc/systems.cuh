// systems.cuh -- small-state ODE systems for the fused Newton kernels.
//
// Each system describes the explicit Euler step map phi(x) = x + h f(x)
// (eq. 2.2) through
//   eval(xp, xc, r, jv):  r  = xc - phi(xp)            (one entry of h(xi), eq. 3.8)
//                         jv = the entries of J = dphi/dx(xp) = I + h df/dx(xp)
//                              that depend on xp (a compact Jacobian)
//   jmul(jv, M, out):     out = J M   (M, out: D x D row-major)
//   jvec(jv, v, out):     out = J v
//   jvec_sub(jv, v, r, out): out = J v - r (fused)
//   jtvec(jv, v, out):    out = J^T v           (adjoint)
//   vjp_param(xp, v, g):  g += (dphi/dp(xp))^T v  (adjoint, g has P entries)
//   jac(xp, jv):          the compact Jacobian alone
//   eval_mixed(xp, xc, r, sv), sfull(sv, S): FP64 residual with the compact
//                         Jacobian in FP32 delta form S = J - I (mixed scan),
//                         the latter computed in FP32 from the states rounded
//                         on the integer pipes (no FP64-pipe work for it)
//   jfull(jv, J):         the dense D x D Jacobian from its compact form
//   eval_ff(xp, xc, r, jv), leaf_ff(jv, r, P, c), replay_ff(jv, r, z),
//   jfull_ff(jv, J):      FP64 residual with the compact Jacobian in
//                         float-float (ffarith.cuh), the fold of one leaf
//                         (P, c) <- (J P, J c - r), the replay z <- J z - r,
//                         and the dense Jacobian, in float-float
// The compact form stores only the state-dependent entries of J, so an
// element of the scan costs D + JN registers instead of D + D*D.
#pragma once

#include <type_traits>

#include "ffarith.cuh"
#include "fpconv.cuh"

namespace pitn {

// Lorenz-63: f = (s(y-x), x(r-z)-y, xy-b z).
//   J = [[1-hs, hs, 0], [h(r-z), 1-h, -hx], [hy, hx, 1-hb]]
struct Lorenz63 {
    static constexpr int D = 3, JN = 3, P = 3;
    double s, r, b, h;
    double j00, j01, j11, j22;
    float hs_f, h_f, hb_f, r_f;
    __host__ __device__ void init(const double* p, double hh) {
        s = p[0]; r = p[1]; b = p[2]; h = hh;
        j00 = 1.0 - h * s; j01 = h * s; j11 = 1.0 - h; j22 = 1.0 - h * b;
        hs_f = (float)(h * s); h_f = (float)h; hb_f = (float)(h * b); r_f = (float)r;
    }
    __device__ __forceinline__ void eval(const double* xp, const double* xc, double* res,
                                         double* jv) const {
        double f0 = s * (xp[1] - xp[0]);
        double f1 = xp[0] * (r - xp[2]) - xp[1];
        double f2 = xp[0] * xp[1] - b * xp[2];
        res[0] = xc[0] - (xp[0] + h * f0);
        res[1] = xc[1] - (xp[1] + h * f1);
        res[2] = xc[2] - (xp[2] + h * f2);
        jv[0] = h * (r - xp[2]);
        jv[1] = h * xp[0];
        jv[2] = h * xp[1];
    }
    __device__ __forceinline__ void jmul(const double* jv, const double* M, double* o) const {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double m0 = M[j], m1 = M[3 + j], m2 = M[6 + j];
            o[j] = j00 * m0 + j01 * m1;
            o[3 + j] = jv[0] * m0 + j11 * m1 - jv[1] * m2;
            o[6 + j] = jv[2] * m0 + jv[1] * m1 + j22 * m2;
        }
    }
    __device__ __forceinline__ void jvec(const double* jv, const double* v, double* o) const {
        double v0 = v[0], v1 = v[1], v2 = v[2];
        o[0] = j00 * v0 + j01 * v1;
        o[1] = jv[0] * v0 + j11 * v1 - jv[1] * v2;
        o[2] = jv[2] * v0 + jv[1] * v1 + j22 * v2;
    }
    // o = J v - r
    __device__ __forceinline__ void jvec_sub(const double* jv, const double* v, const double* rr,
                                             double* o) const {
        double v0 = v[0], v1 = v[1], v2 = v[2];
        o[0] = fma(j00, v0, fma(j01, v1, -rr[0]));
        o[1] = fma(jv[0], v0, fma(j11, v1, fma(-jv[1], v2, -rr[1])));
        o[2] = fma(jv[2], v0, fma(jv[1], v1, fma(j22, v2, -rr[2])));
    }
    __device__ __forceinline__ void jtvec(const double* jv, const double* v, double* o) const {
        double v0 = v[0], v1 = v[1], v2 = v[2];
        o[0] = j00 * v0 + jv[0] * v1 + jv[2] * v2;
        o[1] = j01 * v0 + j11 * v1 + jv[1] * v2;
        o[2] = -jv[1] * v1 + j22 * v2;
    }
    // mixed precision: FP64 residual, FP32 delta form S = J - I
    __device__ __forceinline__ void eval_mixed(const double* xp, const double* xc, double* res,
                                               float* sv) const {
        const double f0 = s * (xp[1] - xp[0]);
        const double f1 = xp[0] * (r - xp[2]) - xp[1];
        const double f2 = xp[0] * xp[1] - b * xp[2];
        res[0] = xc[0] - (xp[0] + h * f0);
        res[1] = xc[1] - (xp[1] + h * f1);
        res[2] = xc[2] - (xp[2] + h * f2);
        const float xf = d2f_int(xp[0]), yf = d2f_int(xp[1]), zf = d2f_int(xp[2]);
        sv[0] = h_f * (r_f - zf);
        sv[1] = h_f * xf;
        sv[2] = h_f * yf;
    }
    __device__ __forceinline__ void sfull(const float* sv, float* S) const {
        S[0] = -hs_f; S[1] = hs_f;  S[2] = 0.f;
        S[3] = sv[0]; S[4] = -h_f;  S[5] = -sv[1];
        S[6] = sv[2]; S[7] = sv[1]; S[8] = -hb_f;
    }
    __device__ __forceinline__ void jfull(const double* jv, double* J) const {
        J[0] = j00;   J[1] = j01;   J[2] = 0.0;
        J[3] = jv[0]; J[4] = j11;   J[5] = -jv[1];
        J[6] = jv[2]; J[7] = jv[1]; J[8] = j22;
    }
    // float-float scan: constants split once per solve (for one IVP on the
    // host, for each IVP of a batch on the device), fc = (h, h rho,
    // 1 - h sigma, h sigma, 1 - h, 1 - h beta) as hi/lo pairs
    ff h_ff, hr_ff, j00_ff, j01_ff, j11_ff, j22_ff;
    __host__ __device__ static void ff_consts(const double* p, double hh, float* fc, double* dc) {
        const double c[6] = {hh, hh * p[1], 1.0 - hh * p[0], hh * p[0], 1.0 - hh, 1.0 - hh * p[2]};
        for (int i = 0; i < 6; ++i) {
            const ff v = ff_const(c[i]);
            fc[2 * i] = v.hi;
            fc[2 * i + 1] = v.lo;
        }
        (void)dc;
    }
    __device__ __forceinline__ void init_ff(const float* fc, const double*) {
        h_ff = ff{fc[0], fc[1]};
        hr_ff = ff{fc[2], fc[3]};
        j00_ff = ff{fc[4], fc[5]};
        j01_ff = ff{fc[6], fc[7]};
        j11_ff = ff{fc[8], fc[9]};
        j22_ff = ff{fc[10], fc[11]};
    }
    // FP64 residual (as eval); compact Jacobian jv = (h (rho - z), h x, h y)
    // in float-float from the states split on the integer pipes
    __device__ __forceinline__ void eval_ff(const double* xp, const double* xc, double* res, ff* jv) const {
        const double f0 = s * (xp[1] - xp[0]);
        const double f1 = xp[0] * (r - xp[2]) - xp[1];
        const double f2 = xp[0] * xp[1] - b * xp[2];
        res[0] = xc[0] - (xp[0] + h * f0);
        res[1] = xc[1] - (xp[1] + h * f1);
        res[2] = xc[2] - (xp[2] + h * f2);
        const ff xf = ff_from_double(xp[0]), yf = ff_from_double(xp[1]), zf = ff_from_double(xp[2]);
        jv[0] = ff_sub(hr_ff, ff_mul(h_ff, zf));
        jv[1] = ff_mul(h_ff, xf);
        jv[2] = ff_mul(h_ff, yf);
    }
    // o = J v, J = [[j00, j01, 0], [jv0, j11, -jv1], [jv2, jv1, j22]]
    __device__ __forceinline__ void jvec_ff(const ff* jv, const ff* v, ff* o) const {
        const ff v0 = v[0], v1 = v[1], v2 = v[2];
        o[0] = ff_fma(j00_ff, v0, ff_mul(j01_ff, v1));
        o[1] = ff_fma(jv[0], v0, ff_fma(j11_ff, v1, ff_neg(ff_mul(jv[1], v2))));
        o[2] = ff_fma(jv[2], v0, ff_fma(jv[1], v1, ff_mul(j22_ff, v2)));
    }
    __device__ __forceinline__ void leaf_ff(const ff* jv, const ff* rr, ff* Pm, ff* c) const {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const ff col[3] = {Pm[j], Pm[3 + j], Pm[6 + j]};
            ff o[3];
            jvec_ff(jv, col, o);
            Pm[j] = o[0];
            Pm[3 + j] = o[1];
            Pm[6 + j] = o[2];
        }
        ff o[3];
        jvec_ff(jv, c, o);
#pragma unroll
        for (int i = 0; i < 3; ++i) c[i] = ff_sub(o[i], rr[i]);
    }
    __device__ __forceinline__ void replay_ff(const ff* jv, const ff* rr, ff* z) const {
        ff o[3];
        jvec_ff(jv, z, o);
#pragma unroll
        for (int i = 0; i < 3; ++i) z[i] = ff_sub(o[i], rr[i]);
    }
    __device__ __forceinline__ void jfull_ff(const ff* jv, ff* J) const {
        J[0] = j00_ff; J[1] = j01_ff; J[2] = ff_zero();
        J[3] = jv[0];  J[4] = j11_ff; J[5] = ff_neg(jv[1]);
        J[6] = jv[2];  J[7] = jv[1];  J[8] = j22_ff;
    }
    __device__ __forceinline__ void jac(const double* xp, double* jv) const {
        jv[0] = h * (r - xp[2]);
        jv[1] = h * xp[0];
        jv[2] = h * xp[1];
    }
    __device__ __forceinline__ void vjp_param(const double* xp, const double* v, double* g) const {
        g[0] += h * (xp[1] - xp[0]) * v[0];
        g[1] += h * xp[0] * v[1];
        g[2] += -h * xp[2] * v[2];
    }
};

// Van der Pol, state (x, v): f = (v, mu(1-x^2)v - x).
//   J = [[1, h], [h(-2 mu x v - 1), 1 + h mu (1-x^2)]]
struct VanDerPol {
    static constexpr int D = 2, JN = 2, P = 1;
    double mu, h, hmu, m2hmu;
    float h_f, hmu_f, m2hmu_f;
    ff h_ff, hmu_ff, m2hmu_ff;
    __host__ __device__ void init(const double* p, double hh) {
        mu = p[0]; h = hh; hmu = h * mu; m2hmu = -2.0 * h * mu;
        h_f = (float)h; hmu_f = (float)hmu; m2hmu_f = (float)m2hmu;
        h_ff = ff_const(h); hmu_ff = ff_const(hmu); m2hmu_ff = ff_const(m2hmu);
    }
    // float-float constants, split once per solve: fc = (h, h mu, -2 h mu)
    // as hi/lo pairs, dc = (h mu, -2 h mu)
    __host__ __device__ static void ff_consts(const double* p, double hh, float* fc, double* dc) {
        const double c[3] = {hh, hh * p[0], -2.0 * hh * p[0]};
        for (int i = 0; i < 3; ++i) {
            const ff v = ff_const(c[i]);
            fc[2 * i] = v.hi;
            fc[2 * i + 1] = v.lo;
        }
        dc[0] = c[1];
        dc[1] = c[2];
    }
    __device__ __forceinline__ void init_ff(const float* fc, const double* dc) {
        h_ff = ff{fc[0], fc[1]};
        hmu_ff = ff{fc[2], fc[3]};
        m2hmu_ff = ff{fc[4], fc[5]};
        hmu = dc[0];
        m2hmu = dc[1];
    }
    // float-float scan: FP64 residual (as eval), J = [[1, h], [a, b]] with
    // a = -2 h mu x v - h and b = 1 + h mu (1 - x^2) in float-float from the
    // states split on the integer pipes
    __device__ __forceinline__ void eval_ff(const double* xp, const double* xc, double* res, ff* jv) const {
        const double x = xp[0], v = xp[1];
        const double w = fma(-x, x, 1.0);
        const double t = hmu * w;
        res[0] = fma(-h, v, xc[0] - x);
        res[1] = fma(h, x, fma(-t, v, xc[1] - v));
        const ff xf = ff_from_double(x), vf = ff_from_double(v);
        jv[0] = ff_sub(ff_mul(ff_mul(m2hmu_ff, xf), vf), h_ff);
        jv[1] = ff_add(ff_one(), ff_mul(hmu_ff, ff_sub(ff_one(), ff_mul(xf, xf))));
    }
    // (P, c) <- (J P, J c - r)
    __device__ __forceinline__ void leaf_ff(const ff* jv, const ff* r, ff* Pm, ff* c) const {
        const ff p00 = Pm[0], p01 = Pm[1], p10 = Pm[2], p11 = Pm[3];
        Pm[0] = ff_fma(h_ff, p10, p00);
        Pm[1] = ff_fma(h_ff, p11, p01);
        Pm[2] = ff_fma(jv[0], p00, ff_mul(jv[1], p10));
        Pm[3] = ff_fma(jv[0], p01, ff_mul(jv[1], p11));
        const ff c0 = c[0], c1 = c[1];
        c[0] = ff_sub(ff_fma(h_ff, c1, c0), r[0]);
        c[1] = ff_sub(ff_fma(jv[0], c0, ff_mul(jv[1], c1)), r[1]);
    }
    // z <- J z - r
    __device__ __forceinline__ void replay_ff(const ff* jv, const ff* r, ff* z) const {
        const ff z0 = z[0], z1 = z[1];
        z[0] = ff_sub(ff_fma(h_ff, z1, z0), r[0]);
        z[1] = ff_sub(ff_fma(jv[0], z0, ff_mul(jv[1], z1)), r[1]);
    }
    __device__ __forceinline__ void jfull_ff(const ff* jv, ff* J) const {
        J[0] = ff_one(); J[1] = h_ff;
        J[2] = jv[0];    J[3] = jv[1];
    }
    // r = xc - x - h f(x) written as r0 = (xc0 - x) - h v,
    // r1 = (xc1 - v) - (h mu w) v + h x with w = 1 - x^2; 10 FP64 operations
    __device__ __forceinline__ void eval(const double* xp, const double* xc, double* res,
                                         double* jv) const {
        const double x = xp[0], v = xp[1];
        const double w = fma(-x, x, 1.0);
        const double t = hmu * w;
        res[0] = fma(-h, v, xc[0] - x);
        res[1] = fma(h, x, fma(-t, v, xc[1] - v));
        jv[0] = fma(m2hmu * x, v, -h);
        jv[1] = 1.0 + t;
    }
    // o = J v - r
    __device__ __forceinline__ void jvec_sub(const double* jv, const double* v, const double* rr,
                                             double* o) const {
        const double v0 = v[0], v1 = v[1];
        o[0] = fma(h, v1, v0 - rr[0]);
        o[1] = fma(jv[0], v0, fma(jv[1], v1, -rr[1]));
    }
    // mixed precision: FP64 residual, FP32 delta form S = J - I = [[0, h], [a, h mu w]]
    __device__ __forceinline__ void eval_mixed(const double* xp, const double* xc, double* res,
                                               float* sv) const {
        const double x = xp[0], v = xp[1];
        const double w = fma(-x, x, 1.0);
        const double t = hmu * w;
        res[0] = fma(-h, v, xc[0] - x);
        res[1] = fma(h, x, fma(-t, v, xc[1] - v));
        const float xf = d2f_int(x), vf = d2f_int(v);
        sv[0] = fmaf(m2hmu_f * xf, vf, -h_f);
        sv[1] = hmu_f * fmaf(-xf, xf, 1.f);
    }
    __device__ __forceinline__ void sfull(const float* sv, float* S) const {
        S[0] = 0.f; S[1] = h_f;
        S[2] = sv[0]; S[3] = sv[1];
    }
    __device__ __forceinline__ void jmul(const double* jv, const double* M, double* o) const {
        double m00 = M[0], m01 = M[1], m10 = M[2], m11 = M[3];
        o[0] = m00 + h * m10;
        o[1] = m01 + h * m11;
        o[2] = jv[0] * m00 + jv[1] * m10;
        o[3] = jv[0] * m01 + jv[1] * m11;
    }
    __device__ __forceinline__ void jvec(const double* jv, const double* v, double* o) const {
        double v0 = v[0], v1 = v[1];
        o[0] = v0 + h * v1;
        o[1] = jv[0] * v0 + jv[1] * v1;
    }
    __device__ __forceinline__ void jtvec(const double* jv, const double* v, double* o) const {
        double v0 = v[0], v1 = v[1];
        o[0] = v0 + jv[0] * v1;
        o[1] = h * v0 + jv[1] * v1;
    }
    __device__ __forceinline__ void jfull(const double* jv, double* J) const {
        J[0] = 1.0;   J[1] = h;
        J[2] = jv[0]; J[3] = jv[1];
    }
    __device__ __forceinline__ void jac(const double* xp, double* jv) const {
        const double x = xp[0], v = xp[1];
        jv[0] = h * (-2.0 * mu * x * v - 1.0);
        jv[1] = 1.0 + h * mu * (1.0 - x * x);
    }
    __device__ __forceinline__ void vjp_param(const double* xp, const double* v, double* g) const {
        g[0] += h * (1.0 - xp[0] * xp[0]) * xp[1] * v[1];
    }
};

// Damped linear oscillator, state (x, v): f = (v, -w^2 x - 2 z w v); J is constant.
struct LinearOsc {
    static constexpr int D = 2, JN = 1, P = 2;  // JN = 1 keeps arrays non-empty
    double w, z, h, j10, j11, ww, zw2;
    float h_f, j10_f, s11_f;
    ff h_ff, j10_ff, j11_ff;
    __host__ __device__ void init(const double* p, double hh) {
        w = p[0]; z = p[1]; h = hh;
        j10 = -h * w * w; j11 = 1.0 - 2.0 * h * z * w;
        h_f = (float)h; j10_f = (float)j10; s11_f = (float)(-2.0 * h * z * w);
        h_ff = ff_const(h); j10_ff = ff_const(j10); j11_ff = ff_const(j11);
        ww = w * w; zw2 = 2.0 * z * w;
    }
    // float-float constants, split once per solve: fc = (h, j10, j11) as hi/lo
    // pairs, dc = (w^2, 2 z w)
    __host__ __device__ static void ff_consts(const double* p, double hh, float* fc, double* dc) {
        const double c[3] = {hh, -hh * p[0] * p[0], 1.0 - 2.0 * hh * p[1] * p[0]};
        for (int i = 0; i < 3; ++i) {
            const ff v = ff_const(c[i]);
            fc[2 * i] = v.hi;
            fc[2 * i + 1] = v.lo;
        }
        dc[0] = p[0] * p[0];
        dc[1] = 2.0 * p[1] * p[0];
    }
    __device__ __forceinline__ void init_ff(const float* fc, const double* dc) {
        h_ff = ff{fc[0], fc[1]};
        j10_ff = ff{fc[2], fc[3]};
        j11_ff = ff{fc[4], fc[5]};
        ww = dc[0];
        zw2 = dc[1];
    }
    // FP64 residual r = xc - (x + h f(x)), f = (v, -w^2 x - 2 z w v)
    __device__ __forceinline__ void eval_ff(const double* xp, const double* xc, double* res, ff* jv) const {
        const double f1 = fma(-ww, xp[0], -zw2 * xp[1]);
        res[0] = xc[0] - fma(h, xp[1], xp[0]);
        res[1] = xc[1] - fma(h, f1, xp[1]);
        jv[0] = ff_zero();
    }
    __device__ __forceinline__ void leaf_ff(const ff*, const ff* r, ff* Pm, ff* c) const {
        const ff p00 = Pm[0], p01 = Pm[1], p10 = Pm[2], p11 = Pm[3];
        Pm[0] = ff_fma(h_ff, p10, p00);
        Pm[1] = ff_fma(h_ff, p11, p01);
        Pm[2] = ff_fma(j10_ff, p00, ff_mul(j11_ff, p10));
        Pm[3] = ff_fma(j10_ff, p01, ff_mul(j11_ff, p11));
        const ff c0 = c[0], c1 = c[1];
        c[0] = ff_sub(ff_fma(h_ff, c1, c0), r[0]);
        c[1] = ff_sub(ff_fma(j10_ff, c0, ff_mul(j11_ff, c1)), r[1]);
    }
    __device__ __forceinline__ void replay_ff(const ff*, const ff* r, ff* zz) const {
        const ff z0 = zz[0], z1 = zz[1];
        zz[0] = ff_sub(ff_fma(h_ff, z1, z0), r[0]);
        zz[1] = ff_sub(ff_fma(j10_ff, z0, ff_mul(j11_ff, z1)), r[1]);
    }
    __device__ __forceinline__ void jfull_ff(const ff*, ff* J) const {
        J[0] = ff_one(); J[1] = h_ff;
        J[2] = j10_ff;   J[3] = j11_ff;
    }
    __device__ __forceinline__ void eval(const double* xp, const double* xc, double* res,
                                         double* jv) const {
        double f1 = -w * w * xp[0] - 2.0 * z * w * xp[1];
        res[0] = xc[0] - (xp[0] + h * xp[1]);
        res[1] = xc[1] - (xp[1] + h * f1);
        jv[0] = 0.0;
    }
    __device__ __forceinline__ void jmul(const double*, const double* M, double* o) const {
        double m00 = M[0], m01 = M[1], m10 = M[2], m11 = M[3];
        o[0] = m00 + h * m10;
        o[1] = m01 + h * m11;
        o[2] = j10 * m00 + j11 * m10;
        o[3] = j10 * m01 + j11 * m11;
    }
    __device__ __forceinline__ void jvec(const double*, const double* v, double* o) const {
        double v0 = v[0], v1 = v[1];
        o[0] = v0 + h * v1;
        o[1] = j10 * v0 + j11 * v1;
    }
    __device__ __forceinline__ void jvec_sub(const double*, const double* v, const double* rr,
                                             double* o) const {
        const double v0 = v[0], v1 = v[1];
        o[0] = fma(h, v1, v0 - rr[0]);
        o[1] = fma(j10, v0, fma(j11, v1, -rr[1]));
    }
    __device__ __forceinline__ void eval_mixed(const double* xp, const double* xc, double* res,
                                               float* sv) const {
        double jv[1];
        eval(xp, xc, res, jv);
        sv[0] = 0.f;
    }
    __device__ __forceinline__ void sfull(const float*, float* S) const {
        S[0] = 0.f; S[1] = h_f;
        S[2] = j10_f; S[3] = s11_f;
    }
    __device__ __forceinline__ void jtvec(const double*, const double* v, double* o) const {
        double v0 = v[0], v1 = v[1];
        o[0] = v0 + j10 * v1;
        o[1] = h * v0 + j11 * v1;
    }
    __device__ __forceinline__ void jfull(const double*, double* J) const {
        J[0] = 1.0; J[1] = h;
        J[2] = j10; J[3] = j11;
    }
    __device__ __forceinline__ void jac(const double*, double* jv) const { jv[0] = 0.0; }
    __device__ __forceinline__ void vjp_param(const double* xp, const double* v, double* g) const {
        g[0] += h * (-2.0 * w * xp[0] - 2.0 * z * xp[1]) * v[1];
        g[1] += h * (-2.0 * w * xp[1]) * v[1];
    }
};

}  // namespace pitn

// ---------------------------------------------------------------------------
// Classical four-stage Runge-Kutta step map (eq. 2.3, tableau a21 = a32 = 1/2,
// a43 = 1, b = (1/6, 1/3, 1/3, 1/6)) over a right-hand side Rhs, with its
// Jacobian by the chain rule through the stages:
//   K_1 = Jf(x),  K_i = Jf(y_i) (I + h a_{i,i-1} K_{i-1}),
//   dphi/dx = I + h sum_i b_i K_i.
// Rhs provides D, P, init(p), f(x, out), jf(x, J) (dense D x D) and
// jf_times(x, Y, K) = Jf(x) Y written for its own sparsity: a product by a
// structural 0 or 1 of Jf is not an exact no-op in IEEE arithmetic (0 * inf),
// so the compiler keeps it; FP64 instructions are the cost of this map.
// The compact Jacobian of this map is the dense one (JN = D * D).
// ---------------------------------------------------------------------------
namespace pitn {

struct LogisticRhs {
    static constexpr int D = 1, P = 2;
    double r, K;
    __host__ __device__ void init(const double* p) { r = p[0]; K = p[1]; }
    __device__ __forceinline__ void f(const double* x, double* o) const { o[0] = r * x[0] * (1.0 - x[0] / K); }
    __device__ __forceinline__ void jf(const double* x, double* J) const { J[0] = r * (1.0 - 2.0 * x[0] / K); }
    __device__ __forceinline__ void jf_times(const double* x, const double* Y, double* Ko) const {
        double J;
        jf(x, &J);
        Ko[0] = J * Y[0];
    }
};

struct VdpRhs {
    static constexpr int D = 2, P = 1;
    double mu;
    __host__ __device__ void init(const double* p) { mu = p[0]; }
    __device__ __forceinline__ void f(const double* x, double* o) const {
        o[0] = x[1];
        o[1] = mu * (1.0 - x[0] * x[0]) * x[1] - x[0];
    }
    __device__ __forceinline__ void jf(const double* x, double* J) const {
        J[0] = 0.0;
        J[1] = 1.0;
        J[2] = -2.0 * mu * x[0] * x[1] - 1.0;
        J[3] = mu * (1.0 - x[0] * x[0]);
    }
    // Jf = [[0, 1], [a, b]]: the first row of Jf Y is Y's second row
    __device__ __forceinline__ void jf_times(const double* x, const double* Y, double* Ko) const {
        double J[4];
        jf(x, J);
        Ko[0] = Y[2];
        Ko[1] = Y[3];
        Ko[2] = fma(J[3], Y[2], J[2] * Y[0]);
        Ko[3] = fma(J[3], Y[3], J[2] * Y[1]);
    }
    // reduced-precision Jacobian chains of the RK4 map (RK4Map::eval_mixed,
    // eval_ff) are provided
    static constexpr bool kReducedJacobian = true;
    // float-float: the constants the Jacobian needs, (mu, -2 mu)
    __host__ __device__ static void ff_params(const double* p, double* c) {
        c[0] = p[0];
        c[1] = -2.0 * p[0];
    }
    // Jf(y) Y in FP32 (the mixed scan), a = -2 mu y0 y1 - 1, b = mu (1 - y0^2); rc = (mu, -2 mu)
    __device__ __forceinline__ void jf_times_f32(const float* y, const float* Y, float* Ko, const float* rc) const {
        const float a = fmaf(rc[1] * y[0], y[1], -1.f);
        const float b = rc[0] * fmaf(-y[0], y[0], 1.f);
        Ko[0] = Y[2];
        Ko[1] = Y[3];
        Ko[2] = fmaf(b, Y[2], a * Y[0]);
        Ko[3] = fmaf(b, Y[3], a * Y[1]);
    }
    // Jf(y) Y in float-float, a = -2 mu y0 y1 - 1, b = mu (1 - y0^2); rc = (mu, -2 mu)
    __device__ __forceinline__ void jf_times_ff(const ff* y, const ff* Y, ff* Ko, const ff* rc) const {
        const ff a = ff_sub(ff_mul(ff_mul(rc[1], y[0]), y[1]), ff_one());
        const ff b = ff_mul(rc[0], ff_sub(ff_one(), ff_mul(y[0], y[0])));
        Ko[0] = Y[2];
        Ko[1] = Y[3];
        Ko[2] = ff_fma(b, Y[2], ff_mul(a, Y[0]));
        Ko[3] = ff_fma(b, Y[3], ff_mul(a, Y[1]));
    }
};

// Whether a right-hand side provides the reduced-precision Jacobian products
// (jf_times_f32, jf_times_ff, ff_params) that the FP32 and float-float RK4
// chains use: true only where the type says so.
template <class Rhs, class = void>
struct has_reduced_jacobian { static constexpr bool value = false; };
template <class Rhs>
struct has_reduced_jacobian<Rhs, std::void_t<decltype(Rhs::kReducedJacobian)>> {
    static constexpr bool value = Rhs::kReducedJacobian;
};

template <class Rhs>
struct RK4Map {
    static constexpr int D = Rhs::D, JN = D * D, P = Rhs::P;
    Rhs rhs;
    double h;
    // constants of the reduced-precision Jacobian chains (see below): h, h/2,
    // h/6 and the right-hand side's two, as float-float (the FP32 chain uses
    // the high parts); set here for the FP32 scan, from the host's split for
    // the float-float one (init_ff)
    ff h_ff, hh_ff, h6_ff, rc_ff[2];
    __host__ __device__ void init(const double* p, double hh) {
        rhs.init(p);
        h = hh;
        if constexpr (has_reduced_jacobian<Rhs>::value) {
            double rc[2];
            Rhs::ff_params(p, rc);
            h_ff = ff_const(hh);
            hh_ff = ff_const(0.5 * hh);
            h6_ff = ff_const(hh * (1.0 / 6.0));
            rc_ff[0] = ff_const(rc[0]);
            rc_ff[1] = ff_const(rc[1]);
        }
    }
    // r = xc - phi(xp), jv = dphi/dx(xp) (dense, row-major)
    __device__ __forceinline__ void eval(const double* xp, const double* xc, double* res, double* jv) const {
        double k[4][D], Kj[4][D * D], y[D], Y[D * D];
        const double a[4] = {0.0, 0.5, 0.5, 1.0};
        // stage 1 at x itself: K_1 = Jf(x) (the identity factor is not multiplied out)
        rhs.f(xp, k[0]);
        rhs.jf(xp, Kj[0]);
#pragma unroll
        for (int s = 1; s < 4; ++s) {
            const double ha = h * a[s];
#pragma unroll
            for (int i = 0; i < D; ++i) y[i] = fma(ha, k[s - 1][i], xp[i]);
#pragma unroll
            for (int i = 0; i < D * D; ++i)
                Y[i] = (i % (D + 1) == 0) ? fma(ha, Kj[s - 1][i], 1.0) : ha * Kj[s - 1][i];
            rhs.f(y, k[s]);
            rhs.jf_times(y, Y, Kj[s]);
        }
        const double w[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
#pragma unroll
        for (int i = 0; i < D; ++i) {
            double sacc = w[0] * k[0][i];
#pragma unroll
            for (int s = 1; s < 4; ++s) sacc = fma(w[s], k[s][i], sacc);
            res[i] = xc[i] - (xp[i] + h * sacc);
        }
#pragma unroll
        for (int i = 0; i < D * D; ++i) {
            double sacc = w[0] * Kj[0][i];
#pragma unroll
            for (int s = 1; s < 4; ++s) sacc = fma(w[s], Kj[s][i], sacc);
            jv[i] = (i % (D + 1) == 0) ? fma(h, sacc, 1.0) : h * sacc;
        }
    }
    __device__ __forceinline__ void jfull(const double* jv, double* J) const {
#pragma unroll
        for (int i = 0; i < D * D; ++i) J[i] = jv[i];
    }

    // ---- FP32 delta-form scan (PITN_PREC_MIXED_FP32; right-hand sides with
    // ff_params and jf_times_f32) ----
    // The FP64 residual as in eval; S = J - I = (h/6)(K1 + 2 K2 + 2 K3 + K4)
    // (the delta form needs no subtraction here) by the stage chain rule in
    // FP32 from the FP64 stage states rounded on the integer pipes.
    __device__ __forceinline__ void eval_mixed(const double* xp, const double* xc, double* res,
                                               float* sv) const {
        double k[D], ksum[D], y[D];
        float yf[D], Y[D * D], K[D * D], Ks[D * D], rc[2];
        const double a[4] = {0.0, 0.5, 0.5, 1.0};
        const double w[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
        rc[0] = rc_ff[0].hi;
        rc[1] = rc_ff[1].hi;
        rhs.f(xp, k);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            ksum[i] = w[0] * k[i];
            yf[i] = d2f_int(xp[i]);
        }
#pragma unroll
        for (int i = 0; i < D * D; ++i) Y[i] = (i % (D + 1) == 0) ? 1.f : 0.f;
        rhs.jf_times_f32(yf, Y, K, rc);   // K_1 = Jf(x)
#pragma unroll
        for (int i = 0; i < D * D; ++i) Ks[i] = K[i];
#pragma unroll
        for (int s = 1; s < 4; ++s) {
            const double ha = h * a[s];
            const float hs = (s == 3) ? h_ff.hi : hh_ff.hi;
#pragma unroll
            for (int i = 0; i < D; ++i) y[i] = fma(ha, k[i], xp[i]);
#pragma unroll
            for (int i = 0; i < D * D; ++i) Y[i] = (i % (D + 1) == 0) ? fmaf(hs, K[i], 1.f) : hs * K[i];
            rhs.f(y, k);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                ksum[i] = fma(w[s], k[i], ksum[i]);
                yf[i] = d2f_int(y[i]);
            }
            rhs.jf_times_f32(yf, Y, K, rc);
#pragma unroll
            for (int i = 0; i < D * D; ++i) Ks[i] = (s == 3) ? Ks[i] + K[i] : fmaf(2.f, K[i], Ks[i]);
        }
#pragma unroll
        for (int i = 0; i < D; ++i) res[i] = xc[i] - (xp[i] + h * ksum[i]);
#pragma unroll
        for (int i = 0; i < D * D; ++i) sv[i] = h6_ff.hi * Ks[i];
    }
    __device__ __forceinline__ void sfull(const float* sv, float* S) const {
#pragma unroll
        for (int i = 0; i < D * D; ++i) S[i] = sv[i];
    }

    // ---- float-float scan (PITN_PREC_FP64_FF; right-hand sides with
    // ff_params and jf_times_ff) ----
    // The residual is the FP64 one above, operation for operation; the
    // stage chain rule of the Jacobian runs in float-float from the FP64
    // stage states.  Constants split once per solve: (h, h/2, h/6) and the
    // right-hand side's two.
    __host__ __device__ static void ff_consts(const double* p, double hh, float* fc, double* dc) {
        double rc[2];
        Rhs::ff_params(p, rc);
        const double c[5] = {hh, 0.5 * hh, hh / 6.0, rc[0], rc[1]};
        for (int i = 0; i < 5; ++i) {
            const ff v = ff_const(c[i]);
            fc[2 * i] = v.hi;
            fc[2 * i + 1] = v.lo;
        }
        (void)dc;
    }
    __device__ __forceinline__ void init_ff(const float* fc, const double*) {
        h_ff = ff{fc[0], fc[1]};
        hh_ff = ff{fc[2], fc[3]};
        h6_ff = ff{fc[4], fc[5]};
        rc_ff[0] = ff{fc[6], fc[7]};
        rc_ff[1] = ff{fc[8], fc[9]};
    }
    // r = xc - phi(xp) in FP64; jv = dphi/dx(xp) in float-float (dense, row-major)
    __device__ __forceinline__ void eval_ff(const double* xp, const double* xc, double* res, ff* jv) const {
        double k[D], ksum[D], y[D];
        ff yf[D], Y[D * D], K[D * D], Ks[D * D];
        const double a[4] = {0.0, 0.5, 0.5, 1.0};
        const double w[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
        rhs.f(xp, k);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            ksum[i] = w[0] * k[i];
            yf[i] = ff_from_double(xp[i]);
        }
#pragma unroll
        for (int i = 0; i < D * D; ++i) Y[i] = (i % (D + 1) == 0) ? ff_one() : ff_zero();
        rhs.jf_times_ff(yf, Y, K, rc_ff);   // K_1 = Jf(x)
#pragma unroll
        for (int i = 0; i < D * D; ++i) Ks[i] = K[i];
#pragma unroll
        for (int s = 1; s < 4; ++s) {
            const double ha = h * a[s];
            const ff hs = (s == 3) ? h_ff : hh_ff;
#pragma unroll
            for (int i = 0; i < D; ++i) y[i] = fma(ha, k[i], xp[i]);
#pragma unroll
            for (int i = 0; i < D * D; ++i) Y[i] = (i % (D + 1) == 0) ? ff_fma(hs, K[i], ff_one()) : ff_mul(hs, K[i]);
            rhs.f(y, k);
#pragma unroll
            for (int i = 0; i < D; ++i) {
                ksum[i] = fma(w[s], k[i], ksum[i]);
                yf[i] = ff_from_double(y[i]);
            }
            rhs.jf_times_ff(yf, Y, K, rc_ff);
#pragma unroll
            for (int i = 0; i < D * D; ++i) {
                const ff kk = (s == 3) ? K[i] : ff{2.f * K[i].hi, 2.f * K[i].lo};   // 2 K: exact
                Ks[i] = ff_add(Ks[i], kk);
            }
        }
#pragma unroll
        for (int i = 0; i < D; ++i) res[i] = xc[i] - (xp[i] + h * ksum[i]);
#pragma unroll
        for (int i = 0; i < D * D; ++i) jv[i] = (i % (D + 1) == 0) ? ff_fma(h6_ff, Ks[i], ff_one()) : ff_mul(h6_ff, Ks[i]);
    }
    // (P, c) <- (J, -r) o (P, c), eq. 3.3
    __device__ __forceinline__ void leaf_ff(const ff* jv, const ff* r, ff* Pm, ff* c) const {
        ff tP[D * D], tc[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
#pragma unroll
            for (int j = 0; j < D; ++j) {
                ff sacc = ff_mul(jv[i * D], Pm[j]);
#pragma unroll
                for (int l = 1; l < D; ++l) sacc = ff_fma(jv[i * D + l], Pm[l * D + j], sacc);
                tP[i * D + j] = sacc;
            }
            ff sacc = ff_neg(r[i]);
#pragma unroll
            for (int l = 0; l < D; ++l) sacc = ff_fma(jv[i * D + l], c[l], sacc);
            tc[i] = sacc;
        }
#pragma unroll
        for (int i = 0; i < D * D; ++i) Pm[i] = tP[i];
#pragma unroll
        for (int i = 0; i < D; ++i) c[i] = tc[i];
    }
    // z <- J z - r
    __device__ __forceinline__ void replay_ff(const ff* jv, const ff* r, ff* z) const {
        ff t[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            ff sacc = ff_neg(r[i]);
#pragma unroll
            for (int l = 0; l < D; ++l) sacc = ff_fma(jv[i * D + l], z[l], sacc);
            t[i] = sacc;
        }
#pragma unroll
        for (int i = 0; i < D; ++i) z[i] = t[i];
    }
    __device__ __forceinline__ void jfull_ff(const ff* jv, ff* J) const {
#pragma unroll
        for (int i = 0; i < D * D; ++i) J[i] = jv[i];
    }

    __device__ __forceinline__ void jmul(const double* jv, const double* M, double* o) const {
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                double sacc = 0.0;
#pragma unroll
                for (int l = 0; l < D; ++l) sacc = fma(jv[i * D + l], M[l * D + j], sacc);
                o[i * D + j] = sacc;
            }
    }
    __device__ __forceinline__ void jvec(const double* jv, const double* v, double* o) const {
#pragma unroll
        for (int i = 0; i < D; ++i) {
            double sacc = 0.0;
#pragma unroll
            for (int l = 0; l < D; ++l) sacc = fma(jv[i * D + l], v[l], sacc);
            o[i] = sacc;
        }
    }
    __device__ __forceinline__ void jvec_sub(const double* jv, const double* v, const double* rr, double* o) const {
#pragma unroll
        for (int i = 0; i < D; ++i) {
            double sacc = -rr[i];
#pragma unroll
            for (int l = 0; l < D; ++l) sacc = fma(jv[i * D + l], v[l], sacc);
            o[i] = sacc;
        }
    }
};

// Explicit Euler over a right-hand side Rhs with a dense Jacobian
// (phi = x + h f(x), dphi/dx = I + h Jf(x)), for systems without a
// hand-specialised compact form.
template <class Rhs>
struct EulerMap : RK4Map<Rhs> {
    using Base = RK4Map<Rhs>;
    static constexpr int D = Rhs::D, JN = D * D, P = Rhs::P;
    __device__ __forceinline__ void eval(const double* xp, const double* xc, double* res, double* jv) const {
        double fx[D], Jf[D * D];
        this->rhs.f(xp, fx);
        this->rhs.jf(xp, Jf);
#pragma unroll
        for (int i = 0; i < D; ++i) res[i] = xc[i] - (xp[i] + this->h * fx[i]);
#pragma unroll
        for (int i = 0; i < D * D; ++i) jv[i] = ((i % (D + 1) == 0) ? 1.0 : 0.0) + this->h * Jf[i];
    }
};


// Dahlquist test equation (Sec. 4.2): f = lambda y.
struct DahlquistRhs {
    static constexpr int D = 1, P = 1;
    double lam;
    __host__ __device__ void init(const double* p) { lam = p[0]; }
    __device__ __forceinline__ void f(const double* x, double* o) const { o[0] = lam * x[0]; }
    __device__ __forceinline__ void jf(const double*, double* J) const { J[0] = lam; }
};

// Robertson's stiff chemical kinetics (Sec. 4.2), rates {k1, k2, k3}:
//   f = (-k1 y1 + k3 y2 y3,  k1 y1 - k2 y2^2 - k3 y2 y3,  k2 y2^2).
struct RobertsonRhs {
    static constexpr int D = 3, P = 3;
    double k1, k2, k3;
    __host__ __device__ void init(const double* p) { k1 = p[0]; k2 = p[1]; k3 = p[2]; }
    __device__ __forceinline__ void f(const double* x, double* o) const {
        const double a = k1 * x[0], b = k3 * x[1] * x[2], c = k2 * x[1] * x[1];
        o[0] = b - a;
        o[1] = a - c - b;
        o[2] = c;
    }
    __device__ __forceinline__ void jf(const double* x, double* J) const {
        J[0] = -k1;  J[1] = k3 * x[2];                       J[2] = k3 * x[1];
        J[3] = k1;   J[4] = -2.0 * k2 * x[1] - k3 * x[2];    J[5] = -k3 * x[1];
        J[6] = 0.0;  J[7] = 2.0 * k2 * x[1];                 J[8] = 0.0;
    }
};

// Inverse of a D x D matrix (D <= 3, row-major) by the adjugate over the
// determinant: the diagonal blocks I - dg/dx_n of the implicit Newton
// Jacobian are small and, for a step size the rule is used with, well
// conditioned.  A zero determinant gives non-finite entries, which the
// solver's non-finite checks report.
template <int D>
__device__ __forceinline__ void small_inverse(const double* A, double* R) {
    static_assert(D >= 1 && D <= 3, "closed-form inverse for D <= 3");
    if constexpr (D == 1) {
        R[0] = 1.0 / A[0];
    } else if constexpr (D == 2) {
        const double inv = 1.0 / (A[0] * A[3] - A[1] * A[2]);
        R[0] = A[3] * inv;
        R[1] = -A[1] * inv;
        R[2] = -A[2] * inv;
        R[3] = A[0] * inv;
    } else {
        const double c00 = A[4] * A[8] - A[5] * A[7];
        const double c01 = A[5] * A[6] - A[3] * A[8];
        const double c02 = A[3] * A[7] - A[4] * A[6];
        const double inv = 1.0 / (A[0] * c00 + A[1] * c01 + A[2] * c02);
        R[0] = c00 * inv;
        R[1] = (A[2] * A[7] - A[1] * A[8]) * inv;
        R[2] = (A[1] * A[5] - A[2] * A[4]) * inv;
        R[3] = c01 * inv;
        R[4] = (A[0] * A[8] - A[2] * A[6]) * inv;
        R[5] = (A[2] * A[3] - A[0] * A[5]) * inv;
        R[6] = c02 * inv;
        R[7] = (A[1] * A[6] - A[0] * A[7]) * inv;
        R[8] = (A[0] * A[4] - A[1] * A[3]) * inv;
    }
}

// Backward Euler (eq. 2.5), x_n = x_{n-1} + h f(x_n), i.e. g = h f(x_n) in
// eq. 3.14.  Its Newton Jacobian (eq. 3.16) has diagonal blocks
// M_n = I - h Jf(x_n) and sub-diagonal blocks -I, so the Newton step
// (eqs. 3.17-3.19) is the affine recursion
//   dx_n = M_n^{-1} dx_{n-1} - M_n^{-1} h_n,   h_n = x_n - x_{n-1} - h f(x_n),
// with element (M_n^{-1}, -M_n^{-1} h_n).  eval returns r = M_n^{-1} h_n, the
// preconditioned residual (the solver's stopping quantity for this rule,
// whose iteration-0 value from a zero guess is the paper's 1/(1 - h lambda)
// for the Dahlquist test), and the dense M_n^{-1} as the compact Jacobian;
// unlike the explicit maps both depend on x_n as well as x_{n-1}.
template <class Rhs>
struct BackwardEulerMap : RK4Map<Rhs> {
    static constexpr int D = Rhs::D, JN = D * D, P = Rhs::P;
    __device__ __forceinline__ void eval(const double* xp, const double* xc, double* res, double* jv) const {
        double fx[D], M[D * D], hn[D];
        this->rhs.f(xc, fx);
        this->rhs.jf(xc, M);
#pragma unroll
        for (int i = 0; i < D * D; ++i) M[i] = ((i % (D + 1) == 0) ? 1.0 : 0.0) - this->h * M[i];
#pragma unroll
        for (int i = 0; i < D; ++i) hn[i] = xc[i] - xp[i] - this->h * fx[i];
        small_inverse<D>(M, jv);
        this->jvec(jv, hn, res);
    }
    // FP32 delta-form scan (PITN_PREC_MIXED_FP32): the FP64 residual and
    // inverse of eval; the element's S = M_n^{-1} - I formed in FP64 and
    // rounded to FP32 on the integer pipes (dense, row-major)
    __device__ __forceinline__ void eval_mixed(const double* xp, const double* xc, double* res, float* sv) const {
        double Mi[D * D];
        eval(xp, xc, res, Mi);
#pragma unroll
        for (int i = 0; i < D * D; ++i) sv[i] = d2f_int((i % (D + 1) == 0) ? Mi[i] - 1.0 : Mi[i]);
    }
    __device__ __forceinline__ void sfull(const float* sv, float* S) const {
#pragma unroll
        for (int i = 0; i < D * D; ++i) S[i] = sv[i];
    }
    // float-float scan (PITN_PREC_FP64_FF): the FP64 residual and inverse of
    // eval, the element M_n^{-1} split into float-float pairs on the integer
    // pipes; the dense fold, replay and element of RK4Map's float-float
    // helpers.  No constants enter the float-float arithmetic.
    __host__ __device__ static void ff_consts(const double*, double, float*, double*) {}
    __device__ __forceinline__ void init_ff(const float*, const double*) {}
    __device__ __forceinline__ void eval_ff(const double* xp, const double* xc, double* res, ff* jv) const {
        double Mi[D * D];
        eval(xp, xc, res, Mi);
#pragma unroll
        for (int i = 0; i < D * D; ++i) jv[i] = ff_from_double(Mi[i]);
    }
};


// Trapezoidal rule (Sec. 3.4): g = (h/2) (f(x_{n-1}) + f(x_n)).  Now both
// blocks of eq. 3.16 are state dependent: M_n = I - (h/2) Jf(x_n) and the
// sub-diagonal -(I + (h/2) Jf(x_{n-1})), so the scan element of step n is
// (M_n^{-1} (I + (h/2) Jf(x_{n-1})), -M_n^{-1} h_n) (eq. 3.19).
template <class Rhs>
struct TrapezoidMap : RK4Map<Rhs> {
    static constexpr int D = Rhs::D, JN = D * D, P = Rhs::P;
    __device__ __forceinline__ void eval(const double* xp, const double* xc, double* res, double* jv) const {
        double fp[D], fc[D], Jp[D * D], M[D * D], Mi[D * D], hn[D];
        const double w = 0.5 * this->h;
        this->rhs.f(xp, fp);
        this->rhs.f(xc, fc);
        this->rhs.jf(xc, M);
        this->rhs.jf(xp, Jp);
#pragma unroll
        for (int i = 0; i < D * D; ++i) {
            const double e = (i % (D + 1) == 0) ? 1.0 : 0.0;
            M[i] = e - w * M[i];
            Jp[i] = e + w * Jp[i];
        }
#pragma unroll
        for (int i = 0; i < D; ++i) hn[i] = xc[i] - xp[i] - w * (fp[i] + fc[i]);
        small_inverse<D>(M, Mi);
        this->jmul(Mi, Jp, jv);
        this->jvec(Mi, hn, res);
    }
    // the reduced-precision scans, as for backward Euler: the FP64 residual and
    // element of eval; S = J - I rounded to FP32, or J split into float-float
    // pairs, on the integer pipes
    __device__ __forceinline__ void eval_mixed(const double* xp, const double* xc, double* res, float* sv) const {
        double J[D * D];
        eval(xp, xc, res, J);
#pragma unroll
        for (int i = 0; i < D * D; ++i) sv[i] = d2f_int((i % (D + 1) == 0) ? J[i] - 1.0 : J[i]);
    }
    __device__ __forceinline__ void sfull(const float* sv, float* S) const {
#pragma unroll
        for (int i = 0; i < D * D; ++i) S[i] = sv[i];
    }
    __host__ __device__ static void ff_consts(const double*, double, float*, double*) {}
    __device__ __forceinline__ void init_ff(const float*, const double*) {}
    __device__ __forceinline__ void eval_ff(const double* xp, const double* xc, double* res, ff* jv) const {
        double J[D * D];
        eval(xp, xc, res, J);
#pragma unroll
        for (int i = 0; i < D * D; ++i) jv[i] = ff_from_double(J[i]);
    }
};

}  // namespace pitn
