// ff_integrate_lorenz_kahan.cu -- compensated (Kahan) RK4 for Lorenz as packed
// f32x2 pairs with group-uniform constants: the measured workload's
// compensated-accumulation variant.
//
// The compensation must see every rounding of the state, so z stays unshifted
// (each stage forms z - r once more than the shifted plain kernel).  The RK4
// weighted sums are those of the plain packed step (sigma folded into the
// x-component's scales, the y-component carried as A = -k_y); each component's
// update x += sc a is compensated: y = sc a - c, t = x + y, c = (t - x) - y,
// x = t.  The registers hold -c, so every operation is a packed add, sub or fma
// (the f32x2 forms have no negation); the planes hold c.
#include "ff_device.cuh"

namespace ff {

struct LorenzKahanConsts {
    f2 h1, h2, h6, nh1, nh2, nh6, sh1, sh2, sh6, nb;
};

__device__ __forceinline__ void lorenz_rk4_pair_kahan(f2& x, f2& y, f2& z, f2& ncx, f2& ncy, f2& ncz, f2 r,
                                                      const LorenzKahanConsts& c, f2 two) {
    f2 d, A, kz, X, Y, Z, ad, aA, az;
    // stage 1 (A = x (z - r) + y = -k_y)
    d = sub2(y, x);
    A = fma2(x, sub2(z, r), y);
    kz = fma2(x, y, mul2(c.nb, z));
    ad = d; aA = A; az = kz;
    X = fma2(c.sh2, d, x); Y = fma2(c.nh2, A, y); Z = fma2(c.h2, kz, z);
    // stage 2
    d = sub2(Y, X);
    A = fma2(X, sub2(Z, r), Y);
    kz = fma2(X, Y, mul2(c.nb, Z));
    ad = fma2(two, d, ad); aA = fma2(two, A, aA); az = fma2(two, kz, az);
    X = fma2(c.sh2, d, x); Y = fma2(c.nh2, A, y); Z = fma2(c.h2, kz, z);
    // stage 3
    d = sub2(Y, X);
    A = fma2(X, sub2(Z, r), Y);
    kz = fma2(X, Y, mul2(c.nb, Z));
    ad = fma2(two, d, ad); aA = fma2(two, A, aA); az = fma2(two, kz, az);
    X = fma2(c.sh1, d, x); Y = fma2(c.nh1, A, y); Z = fma2(c.h1, kz, z);
    // stage 4
    d = sub2(Y, X);
    A = fma2(X, sub2(Z, r), Y);
    kz = fma2(X, Y, mul2(c.nb, Z));
    ad = add2(ad, d); aA = add2(aA, A); az = add2(az, kz);
    // compensated updates
    f2 u, t;
    u = fma2(c.sh6, ad, ncx); t = add2(x, u); ncx = sub2(u, sub2(t, x)); x = t;
    u = fma2(c.nh6, aA, ncy); t = add2(y, u); ncy = sub2(u, sub2(t, y)); y = t;
    u = fma2(c.h6, az, ncz); t = add2(z, u); ncz = sub2(u, sub2(t, z)); z = t;
}

template <bool PP_R, int NPAIR>
__global__ void __launch_bounds__(512) lorenz_rk4_kahan_x2u_kernel(const __grid_constant__ IntegrateArgs a) {
    constexpr int PPT = 2 * NPAIR;
    int g = 0;
#pragma unroll
    for (int q = 1; q < FF_MAX_GROUPS; ++q)
        if (q < a.n_groups && (int)blockIdx.x >= a.gblk[q]) g = q;
    const int64_t nb = a.gblk[g + 1] - a.gblk[g];
    const int64_t first = a.gstart[g] / PPT, last = a.gend[g] / PPT;
    const float h = a.gh[g], sg = a.p[0], b = a.p[2];
    const float h2 = 0.5f * h, h6 = h * (1.0f / 6.0f);
    LorenzKahanConsts c;
    c.h1 = pack2(h, h);
    c.h2 = pack2(h2, h2);
    c.h6 = pack2(h6, h6);
    c.nh1 = pack2(-h, -h);
    c.nh2 = pack2(-h2, -h2);
    c.nh6 = pack2(-h6, -h6);
    c.sh1 = pack2(sg * h, sg * h);
    c.sh2 = pack2(sg * h2, sg * h2);
    c.sh6 = pack2(sg * h6, sg * h6);
    c.nb = pack2(-b, -b);
    const f2 two = pack2(2.0f, 2.0f);
    const int64_t stride = nb * blockDim.x;
    for (int64_t t = first + warp_major_first(blockIdx.x - a.gblk[g], nb); t < last; t += stride) {
        const int64_t i0 = t * PPT;
        float xs[PPT], ys[PPT], zs[PPT], cx[PPT], cy[PPT], cz[PPT], r[PPT];
        Vec<PPT>::load(a.x + i0, xs);
        Vec<PPT>::load(a.x + a.pitch + i0, ys);
        Vec<PPT>::load(a.x + 2 * a.pitch + i0, zs);
        Vec<PPT>::load(a.comp + i0, cx);
        Vec<PPT>::load(a.comp + a.pitch + i0, cy);
        Vec<PPT>::load(a.comp + 2 * a.pitch + i0, cz);
        if (PP_R) Vec<PPT>::load(a.pparam + i0, r);
        if (float* ck0 = start_checkpoint(a)) {
            Vec<PPT>::store(ck0 + i0, xs);
            Vec<PPT>::store(ck0 + a.pitch + i0, ys);
            Vec<PPT>::store(ck0 + 2 * a.pitch + i0, zs);
        }
        f2 X[NPAIR], Y[NPAIR], Z[NPAIR], NCX[NPAIR], NCY[NPAIR], NCZ[NPAIR], R[NPAIR];
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) {
            const int u = 2 * q, v = 2 * q + 1;
            X[q] = pack2(xs[u], xs[v]);
            Y[q] = pack2(ys[u], ys[v]);
            Z[q] = pack2(zs[u], zs[v]);
            NCX[q] = pack2(-cx[u], -cx[v]);
            NCY[q] = pack2(-cy[u], -cy[v]);
            NCZ[q] = pack2(-cz[u], -cz[v]);
            R[q] = PP_R ? pack2(r[u], r[v]) : pack2(a.p[1], a.p[1]);
        }
        auto save = [&](int slot) {
            // the state is kept unshifted; the compensation stays in registers
            float* ck = a.ckpt + (int64_t)slot * a.ck_stride;
            float sx[PPT], sy[PPT], sz[PPT];
#pragma unroll
            for (int q = 0; q < NPAIR; ++q) {
                unpack2(X[q], sx[2 * q], sx[2 * q + 1]);
                unpack2(Y[q], sy[2 * q], sy[2 * q + 1]);
                unpack2(Z[q], sz[2 * q], sz[2 * q + 1]);
            }
            Vec<PPT>::store(ck + i0, sx);
            Vec<PPT>::store(ck + a.pitch + i0, sy);
            Vec<PPT>::store(ck + 2 * a.pitch + i0, sz);
        };
        run_steps<2>(a, (int)a.n_steps, [&]() {
#pragma unroll
            for (int q = 0; q < NPAIR; ++q) lorenz_rk4_pair_kahan(X[q], Y[q], Z[q], NCX[q], NCY[q], NCZ[q], R[q], c, two);
        }, save);
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) {
            const int u = 2 * q, v = 2 * q + 1;
            unpack2(X[q], xs[u], xs[v]);
            unpack2(Y[q], ys[u], ys[v]);
            unpack2(Z[q], zs[u], zs[v]);
            unpack2(NCX[q], cx[u], cx[v]);
            unpack2(NCY[q], cy[u], cy[v]);
            unpack2(NCZ[q], cz[u], cz[v]);
        }
#pragma unroll
        for (int j = 0; j < PPT; ++j) { cx[j] = -cx[j]; cy[j] = -cy[j]; cz[j] = -cz[j]; }
        Vec<PPT>::store(a.x + i0, xs);
        Vec<PPT>::store(a.x + a.pitch + i0, ys);
        Vec<PPT>::store(a.x + 2 * a.pitch + i0, zs);
        Vec<PPT>::store(a.comp + i0, cx);
        Vec<PPT>::store(a.comp + a.pitch + i0, cy);
        Vec<PPT>::store(a.comp + 2 * a.pitch + i0, cz);
    }
}

bool lorenz_kahan_packed(int method, bool pp, const IntegrateArgs& a, const LaunchShape& shape) {
    if (method != FF_RK4 || a.reset || (shape.ppt != 2 && shape.ppt != 4)) return false;
    for (int g = 0; g < a.n_groups; ++g)
        if (a.gstart[g] % shape.ppt != 0) return false;
    return !pp || a.pidx == 1;
}

cudaError_t launch_integrate_lorenz_kahan(bool pp, const IntegrateArgs& a, const LaunchShape& shape,
                                          cudaStream_t stream) {
    if (shape.ppt == 2)
        return pp ? uniform_launch(lorenz_rk4_kahan_x2u_kernel<true, 1>, a, shape, stream)
                  : uniform_launch(lorenz_rk4_kahan_x2u_kernel<false, 1>, a, shape, stream);
    return pp ? uniform_launch(lorenz_rk4_kahan_x2u_kernel<true, 2>, a, shape, stream)
              : uniform_launch(lorenz_rk4_kahan_x2u_kernel<false, 2>, a, shape, stream);
}

}  // namespace ff
