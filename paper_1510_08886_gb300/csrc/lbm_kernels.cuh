// Device code of the fused stream-collide step (templates, instantiated per
// precision in k_fp64.cu and k_fp32.cu).
//
// One thread owns one lattice node (x, y).  Per time step it
//   1. pulls the V post-collision populations of the previous step from
//      (x - e_x mod Nx, y - e_y), or, where that source lies beyond a wall,
//      fills them from the diffuse-wall flux balance (Eq. nm.14, nm.15);
//   2. forms the moments rho, u (Eq. nm.10) and the momentum flux needed by
//      the force term (Eq. nm.4, with Pi of f from Eq. nm.7);
//   3. relaxes every population towards feq = f0 + tau F
//      (Eq. nm.2, nm.3, nm.8) and writes it to the other lattice.
//
// Populations are stored as deviations d_a = fbar_a - w_a from the rest state
// at rho0 = 1 (exact rewrite: sum w = 1, sum w e = 0, sum w xi xi = delta), so
// every quantity the arithmetic touches is O(Ma): fp32 keeps ~7 significant
// digits of the flow, fp64 gains a few bits over storing fbar.
//
// Velocities come in +-e pairs: the equilibrium and force terms split into
// parts even and odd in e, each evaluated once per pair.
#pragma once

#include <math.h>

#include "lbm_internal.h"

namespace lbm {

template <typename C> __device__ __forceinline__ C cinf();
template <> __device__ __forceinline__ double cinf<double>() { return HUGE_VAL; }
template <> __device__ __forceinline__ float cinf<float>() { return HUGE_VALF; }

// Wall flux balance (Eq. nm.15) for landing column x, in deviation form:
// returns dPsi = sum_out d_b / sum_in |e_y| w  so that an unknown incoming
// population is d_a = dPsi * w_a, i.e. fbar_a = Psi rho_w w_a (Eq. nm.14).
// Outgoing populations b (e_y < 0 at the bottom wall, e_y > 0 at the top)
// cross the wall from their |e_y| rows nearest to it and are credited to the
// column they land on, so the source column is x - e_x.  fp64 accumulation.
template <typename S, typename C>
__device__ __noinline__ double wall_dpsi(const KParams<C>& k, const S* __restrict__ src,
                                         int x, bool bottom) {
    double acc = 0.0;
    for (int b = k.R; b < k.V; ++b) {
        const int ey = k.ey[b];
        if (bottom ? (ey >= 0) : (ey <= 0)) continue;
        int xs = x - k.sx[b];
        xs += (xs < 0) ? k.Nx : 0;
        const int n = bottom ? -ey : ey;
        const S* pl = src + (long long)b * k.plane + xs;
        for (int j = 0; j < n; ++j) {
            const int row = bottom ? j : (k.Ny - 1 - j);
            acc += (double)pl[(long long)row * k.Nx];
        }
    }
    return acc * k.inv_den;
}

// Per-node coefficients of the relaxation target, from the deviation moments
//   drho = sum d, J = sum d e, K = sum d e e  (velocities in units of c).
template <typename C>
struct CellCoef {
    C rho, drho, ux, uy;
    C utx, uty;               // c u: s = u.xi = (c u).e
    C a0, a1, a2;             // even part:  a0 + t (a1 + t a2) [+ tr ge s]
    C b0, b1;                 // odd part:   s (b0 + t b1) [+ force terms]
    C tr;                     // tau rho
    C qxx, qxy, qyy, qtr;     // (tau/2) Q = qxx ex^2 + qxy 2 ex ey + qyy ey^2 - qtr
    C hx, hy;                 // tau (g.A).xi = hx ex + hy ey
};

template <int N, typename C>
__device__ __forceinline__ CellCoef<C> cell_coef(const KParams<C>& k, C drho, C Jx, C Jy,
                                                 C Kxx, C Kxy, C Kyy) {
    CellCoef<C> q;
    q.drho = drho;
    q.rho = C(1) + drho;
    const C inv = C(1) / q.rho;
    // Eq. nm.10: rho u = sum fbar xi + (dt/2) rho g
    q.ux = k.c * Jx * inv + k.hdt * k.gx;
    q.uy = k.c * Jy * inv + k.hdt * k.gy;
    q.utx = k.c * q.ux;
    q.uty = k.c * q.uy;
    const C u2 = q.ux * q.ux + q.uy * q.uy;
    // f0/(rho w) - 1 of Eq. nm.3 (+ the N = 4 Hermite term of Eq. equi.hermite)
    // with s = u.xi, t = s^2:
    //   even: (t - u2)/2 + [N>=4] (t^2 - 6 t u2 + 3 u2^2)/24
    //   odd:  s + [N>=3] s (t - 3 u2)/6
    q.a0 = drho + q.rho * (C(-0.5) * u2 + (N >= 4 ? C(0.125) * u2 * u2 : C(0)));
    q.a1 = q.rho * (C(0.5) - (N >= 4 ? C(0.25) * u2 : C(0)));
    q.a2 = N >= 4 ? q.rho * C(1.0 / 24.0) : C(0);
    q.b0 = q.rho * (N >= 3 ? C(1) - C(0.5) * u2 : C(1));
    q.b1 = N >= 3 ? q.rho * C(1.0 / 6.0) : C(0);
    q.tr = k.tau * q.rho;
    if (k.force) {
        // even force part of Eq. nm.4: tau rho ((g.xi)(u.xi) - u.g)
        q.a0 -= q.tr * (q.ux * k.gx + q.uy * k.gy);
        // A = Pi - rho delta, Pi the momentum flux of f = (2 tau fbar + dt feq)
        // / (2 tau + dt) (Eq. nm.7 inverted), Pibar = delta + c^2 K and
        // Pi_eq = rho (delta + u u + tau (g u + u g)) (exact for Q >= N + 2):
        //   (2 tau + dt) A = -2 tau drho delta + 2 tau c^2 K
        //                    + dt rho (u u + tau (g u + u g))
        const C tdr = k.dt * q.rho;
        const C Axx = (k.two_tau * (k.c2 * Kxx - drho) +
                       tdr * (q.ux * q.ux + C(2) * k.tau * k.gx * q.ux)) * k.inv_2tau_dt;
        const C Ayy = (k.two_tau * (k.c2 * Kyy - drho) +
                       tdr * (q.uy * q.uy + C(2) * k.tau * k.gy * q.uy)) * k.inv_2tau_dt;
        const C Axy = (k.two_tau * k.c2 * Kxy +
                       tdr * (q.ux * q.uy + k.tau * (k.gx * q.uy + k.gy * q.ux))) * k.inv_2tau_dt;
        if (N >= 3) {
            // third-order force term (1/2) A:((g.xi) H2(xi) - 2 g xi)
            q.qxx = k.half_tau * k.c2 * Axx;
            q.qxy = k.half_tau * k.c2 * Axy;   // multiplies 2 ex ey
            q.qyy = k.half_tau * k.c2 * Ayy;
            q.qtr = k.half_tau * (Axx + Ayy);
            q.hx = k.tau * k.c * (k.gx * Axx + k.gy * Axy);
            q.hy = k.tau * k.c * (k.gx * Axy + k.gy * Ayy);
        } else {
            q.qxx = q.qxy = q.qyy = q.qtr = q.hx = q.hy = C(0);
        }
    }
    return q;
}

// Relax one +-e pair (planes fp, fm) in place:
//   d* = (1 - omega) d + omega w (feq/w - 1),  feq/w - 1 = Ge +- Go.
template <bool FORCE, typename C>
__device__ __forceinline__ void pair_update(const KParams<C>& k, const CellCoef<C>& q, int p,
                                            C& fp, C& fm) {
    const C ex = k.pex[p], ey = k.pey[p];
    const C s = fma(q.uty, ey, q.utx * ex);
    const C t = s * s;
    C Ge = fma(t, fma(t, q.a2, q.a1), q.a0);
    C Go = s * fma(t, q.b1, q.b0);
    if (FORCE) {
        const C ge = k.pge[p];
        // odd force part: tau rho (g.xi) + (tau/2)((g.xi) Q - 2 (g.A).xi)
        const C halfQ = fma(q.qxx, k.pexx[p], fma(q.qxy, k.pexy2[p], fma(q.qyy, k.peyy[p], -q.qtr)));
        Ge = fma(q.tr * ge, s, Ge);
        Go = fma(ge, q.tr + halfQ, Go) - fma(q.hx, ex, q.hy * ey);
    }
    const C X = k.pomw[p] * Ge, Y = k.pomw[p] * Go;
    fp = fma(k.one_m_omega, fp, X + Y);
    fm = fma(k.one_m_omega, fm, X - Y);
}

template <typename C>
__device__ __forceinline__ void flag_density(const CellCoef<C>& q, unsigned int* status) {
    if (!(q.rho > C(0) && q.rho < cinf<C>())) atomicOr(status, 1u);
}

template <typename C>
__device__ __forceinline__ void emit_moments(const KParams<C>& k, const CellCoef<C>& q, int cell,
                                             const DevBufs& b) {
    if (k.emit) {
        b.rho[cell] = 1.0 + (double)q.drho;
        b.ux[cell] = (double)q.ux;
        b.uy[cell] = (double)q.uy;
    }
}

// Pull one population of plane a into node (x, y) of an interior row.
template <typename S, typename C>
__device__ __forceinline__ C pull(const KParams<C>& k, const S* __restrict__ src, int a, int x, int y) {
    int xs = x - k.sx[a];
    xs += (xs < 0) ? k.Nx : 0;
    return C(src[(long long)a * k.plane + (long long)(y - k.ey[a]) * k.Nx + xs]);
}

// Fused step for a DVM with R rest planes and P pairs known at compile time:
// the V populations stay in registers between the moment pass and the
// relaxation pass.
template <int R, int P, int N, typename S, typename C>
__global__ void __launch_bounds__(kBlock)
k_step(const __grid_constant__ KParams<C> k, const S* __restrict__ src, S* __restrict__ dst,
       const DevBufs b) {
    constexpr int V = R + 2 * P;
    const int cell = blockIdx.x * kBlock + threadIdx.x;
    if (cell >= k.ncell) return;
    const int y = cell / k.Nx;
    const int x = cell - y * k.Nx;
    C f[V];
    const bool nb = y < k.maxey, nt = y >= k.Ny - k.maxey;
    if (!(nb || nt)) {
#pragma unroll
        for (int a = 0; a < V; ++a) f[a] = pull<S, C>(k, src, a, x, y);
    } else {
        const double pb = nb ? wall_dpsi<S, C>(k, src, x, true) : 0.0;
        const double pt = nt ? wall_dpsi<S, C>(k, src, x, false) : 0.0;
#pragma unroll
        for (int a = 0; a < V; ++a) {
            const int ys = y - k.ey[a];
            if (ys < 0)
                f[a] = C(pb * k.w[a]);
            else if (ys >= k.Ny)
                f[a] = C(pt * k.w[a]);
            else
                f[a] = pull<S, C>(k, src, a, x, y);
        }
    }
    // moments of the deviations
    C drho = R ? f[0] : C(0), Jx = 0, Jy = 0, Kxx = 0, Kxy = 0, Kyy = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const C sum = f[R + p] + f[R + P + p], dif = f[R + p] - f[R + P + p];
        drho += sum;
        Jx = fma(k.pex[p], dif, Jx);
        Jy = fma(k.pey[p], dif, Jy);
        Kxx = fma(k.pexx[p], sum, Kxx);
        Kxy = fma(k.pexy2[p], sum, Kxy);
        Kyy = fma(k.peyy[p], sum, Kyy);
    }
    const CellCoef<C> q = cell_coef<N, C>(k, drho, Jx, Jy, Kxx, C(0.5) * Kxy, Kyy);
    if (R) f[0] = fma(k.one_m_omega, f[0], k.omw_rest * q.a0);
    if (k.force) {
#pragma unroll
        for (int p = 0; p < P; ++p) pair_update<true, C>(k, q, p, f[R + p], f[R + P + p]);
    } else {
#pragma unroll
        for (int p = 0; p < P; ++p) pair_update<false, C>(k, q, p, f[R + p], f[R + P + p]);
    }
#pragma unroll
    for (int a = 0; a < V; ++a) dst[(long long)a * k.plane + cell] = S(f[a]);
    emit_moments<C>(k, q, cell, b);
    flag_density<C>(q, b.status);
}

// Same step for any V <= LBM_MAX_V (R, P at run time).  The populations are
// read twice (moment pass, relaxation pass); the second read hits L1/L2.
// INIT = true builds the state from a density field instead of streaming:
// fbar_a = rho0 w_a, then the same relaxation.
template <int N, bool INIT, typename S, typename C>
__global__ void __launch_bounds__(kBlock)
k_generic(const __grid_constant__ KParams<C> k, const S* __restrict__ src,
          const double* __restrict__ rho0, S* __restrict__ dst, const DevBufs b) {
    const int cell = blockIdx.x * kBlock + threadIdx.x;
    if (cell >= k.ncell) return;
    const int y = cell / k.Nx;
    const int x = cell - y * k.Nx;
    double pb = 0.0, pt = 0.0, r0 = 0.0;
    if (INIT) {
        r0 = rho0[cell] - 1.0;
    } else {
        if (y < k.maxey) pb = wall_dpsi<S, C>(k, src, x, true);
        if (y >= k.Ny - k.maxey) pt = wall_dpsi<S, C>(k, src, x, false);
    }
    auto value = [&](int a) -> C {
        if (INIT) return C(r0 * k.w[a]);
        const int ys = y - k.ey[a];
        if (ys < 0) return C(pb * k.w[a]);
        if (ys >= k.Ny) return C(pt * k.w[a]);
        return pull<S, C>(k, src, a, x, y);
    };
    const int R = k.R, P = k.P;
    C drho = R ? value(0) : C(0), Jx = 0, Jy = 0, Kxx = 0, Kxy = 0, Kyy = 0;
    for (int p = 0; p < P; ++p) {
        const C fp = value(R + p), fm = value(R + P + p);
        const C sum = fp + fm, dif = fp - fm;
        drho += sum;
        Jx = fma(k.pex[p], dif, Jx);
        Jy = fma(k.pey[p], dif, Jy);
        Kxx = fma(k.pexx[p], sum, Kxx);
        Kxy = fma(k.pexy2[p], sum, Kxy);
        Kyy = fma(k.peyy[p], sum, Kyy);
    }
    const CellCoef<C> q = cell_coef<N, C>(k, drho, Jx, Jy, Kxx, C(0.5) * Kxy, Kyy);
    if (R) dst[cell] = S(fma(k.one_m_omega, value(0), k.omw_rest * q.a0));
    for (int p = 0; p < P; ++p) {
        C fp = value(R + p), fm = value(R + P + p);
        if (k.force)
            pair_update<true, C>(k, q, p, fp, fm);
        else
            pair_update<false, C>(k, q, p, fp, fm);
        dst[(long long)(R + p) * k.plane + cell] = S(fp);
        dst[(long long)(R + P + p) * k.plane + cell] = S(fm);
    }
    emit_moments<C>(k, q, cell, b);
    flag_density<C>(q, b.status);
}

// Launch helpers -------------------------------------------------------------

template <typename C>
inline dim3 grid_for(const KParams<C>& k) { return dim3((k.ncell + kBlock - 1) / kBlock); }

// Dispatch on (R, P) to a register-resident instantiation, else the generic
// kernel.  Listed shapes: the paper's 2D sets and the (x, z) marginals of its
// 3D sets (V = 16, 32, 33, 37, 40, 41, 48, 53).
template <int N, typename S, typename C>
cudaError_t launch_step_n(const KParams<C>& k, const S* src, S* dst, const DevBufs& b,
                          cudaStream_t st) {
    const dim3 g = grid_for(k);
#define LBM_SHAPE(RR, PP)                                                     \
    if (k.R == RR && k.P == PP) {                                             \
        k_step<RR, PP, N, S, C><<<g, kBlock, 0, st>>>(k, src, dst, b);        \
        return cudaGetLastError();                                            \
    }
    LBM_SHAPE(0, 8)    // 16
    LBM_SHAPE(0, 16)   // 32
    LBM_SHAPE(1, 16)   // 33
    LBM_SHAPE(1, 18)   // 37
    LBM_SHAPE(0, 20)   // 40
    LBM_SHAPE(1, 20)   // 41
    LBM_SHAPE(0, 24)   // 48
    LBM_SHAPE(1, 26)   // 53
#undef LBM_SHAPE
    k_generic<N, false, S, C><<<g, kBlock, 0, st>>>(k, src, nullptr, dst, b);
    return cudaGetLastError();
}

template <typename S, typename C>
cudaError_t launch_step_t(const KParams<C>& k, int N, const void* src, void* dst,
                          const DevBufs& b, cudaStream_t st) {
    const S* s = static_cast<const S*>(src);
    S* d = static_cast<S*>(dst);
    switch (N) {
        case 2: return launch_step_n<2, S, C>(k, s, d, b, st);
        case 3: return launch_step_n<3, S, C>(k, s, d, b, st);
        case 4: return launch_step_n<4, S, C>(k, s, d, b, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename S, typename C>
cudaError_t launch_init_t(const KParams<C>& k, int N, const double* rho0, void* dst,
                          const DevBufs& b, cudaStream_t st) {
    S* d = static_cast<S*>(dst);
    const dim3 g = grid_for(k);
    switch (N) {
        case 2: k_generic<2, true, S, C><<<g, kBlock, 0, st>>>(k, nullptr, rho0, d, b); break;
        case 3: k_generic<3, true, S, C><<<g, kBlock, 0, st>>>(k, nullptr, rho0, d, b); break;
        case 4: k_generic<4, true, S, C><<<g, kBlock, 0, st>>>(k, nullptr, rho0, d, b); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace lbm
