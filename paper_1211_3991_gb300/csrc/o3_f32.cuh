// Single-precision per-spin arithmetic of O(3) spins (App. B names O(3) among
// the continuous models the method carries over to), shared by the plain and
// the resident engines.  Every product, sum and quotient is an explicit
// round-to-nearest intrinsic, so the result does not depend on whether the
// translation unit contracts a * b + c into a fused multiply-add: both
// engines take the same IEEE steps.
#pragma once

#include "device.cuh"

namespace xyl {

__device__ __forceinline__ float o3_dot(float ax, float ay, float az, float bx, float by, float bz)
{
    return __fadd_rn(__fadd_rn(__fmul_rn(ax, bx), __fmul_rn(ay, by)), __fmul_rn(az, bz));
}

// Point of the spherical cap of angular radius half_width around the unit
// vector (x, y, z): 1 - cos theta = u * 2 sin^2(half_width / 2), azimuth
// 2 pi uphi - pi in the frame e1 = (g + x^2 a, b, -x), e2 = (b, g + y^2 a, -y),
// g = sign(z) (+1 at z = 0), a = -1 / (g + z), b = x y a (the orthonormal
// frame of Duff et al., JCGT 2017, first vector times g); the result is
// renormalised.
__device__ __forceinline__ void o3_cap_propose_f32(float x, float y, float z, float half_width, float u, float uphi,
                                                   float &nx, float &ny, float &nz)
{
    float sh, ch;
    __sincosf(__fmul_rn(0.5f, half_width), &sh, &ch);
    const float w = __fmul_rn(u, __fmul_rn(2.0f, __fmul_rn(sh, sh)));
    const float ct = __fsub_rn(1.0f, w);
    const float st = sqrtf(fmaxf(__fmul_rn(w, __fsub_rn(2.0f, w)), 0.0f));
    float sp, cp;
    __sincosf(__fsub_rn(__fmul_rn(6.28318530717958647692f, uphi), 3.14159265358979323846f), &sp, &cp);
    const float g = z >= 0.0f ? 1.0f : -1.0f;
    const float a = __fdiv_rn(-1.0f, __fadd_rn(g, z));
    const float b = __fmul_rn(__fmul_rn(x, y), a);
    const float e1x = __fadd_rn(g, __fmul_rn(__fmul_rn(x, x), a)), e1y = b, e1z = -x;
    const float e2x = b, e2y = __fadd_rn(g, __fmul_rn(__fmul_rn(y, y), a)), e2z = -y;
    const float px = __fadd_rn(__fmul_rn(ct, x), __fmul_rn(st, __fadd_rn(__fmul_rn(cp, e1x), __fmul_rn(sp, e2x))));
    const float py = __fadd_rn(__fmul_rn(ct, y), __fmul_rn(st, __fadd_rn(__fmul_rn(cp, e1y), __fmul_rn(sp, e2y))));
    const float pz = __fadd_rn(__fmul_rn(ct, z), __fmul_rn(st, __fadd_rn(__fmul_rn(cp, e1z), __fmul_rn(sp, e2z))));
    const float inv = rsqrtf(o3_dot(px, py, pz, px, py, pz));
    nx = __fmul_rn(px, inv);
    ny = __fmul_rn(py, inv);
    nz = __fmul_rn(pz, inv);
}

// Metropolis test of the move S -> S' in the local field h: dE = -(S' - S) . h,
// accept iff dE <= 0 or ua < exp(-beta dE).
__device__ __forceinline__ bool o3_accept_f32(float sx, float sy, float sz, float nx, float ny, float nz, float hx,
                                              float hy, float hz, float beta, float ua)
{
    const float dE = -o3_dot(__fsub_rn(nx, sx), __fsub_rn(ny, sy), __fsub_rn(nz, sz), hx, hy, hz);
    return dE <= 0.0f || ua < __expf(__fmul_rn(-beta, dE));
}

// Overrelaxation: S' = 2 (S.h) h / |h|^2 - S; S unchanged when h = 0.
__device__ __forceinline__ void o3_reflect_f32(float sx, float sy, float sz, float hx, float hy, float hz, float &nx,
                                               float &ny, float &nz)
{
    const float h2 = o3_dot(hx, hy, hz, hx, hy, hz);
    if (h2 > 0.0f) {
        const float k = __fdiv_rn(__fmul_rn(2.0f, o3_dot(sx, sy, sz, hx, hy, hz)), h2);
        nx = __fsub_rn(__fmul_rn(k, hx), sx);
        ny = __fsub_rn(__fmul_rn(k, hy), sy);
        nz = __fsub_rn(__fmul_rn(k, hz), sz);
    } else {
        nx = sx;
        ny = sy;
        nz = sz;
    }
}

}  // namespace xyl
