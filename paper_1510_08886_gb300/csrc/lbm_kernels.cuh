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

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <utility>

#include "dvm_sets.h"
#include "lbm_internal.h"

namespace lbm {

template <typename C> __device__ __forceinline__ C cinf();
template <> __device__ __forceinline__ double cinf<double>() { return HUGE_VAL; }
template <> __device__ __forceinline__ float cinf<float>() { return HUGE_VALF; }

// Storage of a population: fp64/fp32 hold the deviation d itself; the 16-bit
// formats hold h = d / (w_a S) so that every plane uses the format's range
// around 1 whatever its weight (d of a plane with w ~ 1e-6 would be subnormal).
//
// 16-bit stores round stochastically: with round-to-nearest the per-step
// relaxation increment of a population is often below half an ulp of h and
// is lost every step, which stalls the flow at a wrong state (2-6 % error in
// the mass flow in fp16).  Adding uniform random bits below the kept mantissa
// and truncating makes every store unbiased.  The random bits are a hash of
// (node, step) advanced by a 32-bit LCG per plane (high bits only), so runs
// are reproducible and a restored checkpoint continues bit for bit.
template <typename S> struct Storage {
    static constexpr bool scaled = false;
};
template <> struct Storage<__half> {
    static constexpr bool scaled = true;
    static __device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half from_f(float v) { return __float2half_rn(v); }
    // fp32 keeps 13 more mantissa bits than fp16
    static __device__ __forceinline__ __half from_f_sr(float v, unsigned r) {
        return __float2half_rz(__uint_as_float(__float_as_uint(v) + (r >> 19)));
    }
};
template <> struct Storage<__nv_bfloat16> {
    static constexpr bool scaled = true;
    static __device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 from_f(float v) { return __float2bfloat16_rn(v); }
    // bf16 is the upper half of fp32
    static __device__ __forceinline__ __nv_bfloat16 from_f_sr(float v, unsigned r) {
        return __ushort_as_bfloat16((unsigned short)((__float_as_uint(v) + (r >> 16)) >> 16));
    }
};

__device__ __forceinline__ unsigned mix32(unsigned x) {   // integer hash (xorshift-multiply)
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

template <typename S, typename C>
__device__ __forceinline__ unsigned sr_seed(unsigned seed, int cell) {
    if constexpr (Storage<S>::scaled) return mix32(unsigned(cell) ^ mix32(seed * 0x9e3779b9u + 1u));
    else return 0u;
}

// Rounded product that the compiler never merges into an add (an FMA).
// Every product in the collision arithmetic that meets an addition is either
// an explicit fma or mul_rn, so each kernel that inlines these functions
// rounds every node identically (no contraction choice is left open).
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Interior population load through the read-only path with a 256-byte L2
// prefetch size: a warp's 128-byte access also brings the next 128 bytes of
// the plane into L2, which the neighbouring warp reads next (measured +0.35 %
// on the 4096 x 512 fp32 step).  16-bit storage takes a plain load.
__device__ __forceinline__ float ld_stream(const float* p) {
    float v;
    asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ double ld_stream(const double* p) {
    double v;
    asm("ld.global.nc.L2::256B.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
template <typename S>
__device__ __forceinline__ S ld_stream(const S* p) {
    return *p;
}

template <typename S, typename C>
__device__ __forceinline__ C ld_pop(const KParams<C>& k, S v, int a) {
    if constexpr (Storage<S>::scaled) return mul_rn(Storage<S>::to_f(v), k.sw[a]);
    else return C(v);
}

template <typename S, typename C>
__device__ __forceinline__ S st_pop(const KParams<C>& k, C v, int a, unsigned& r) {
    if constexpr (Storage<S>::scaled) {
        r = r * 1664525u + 1013904223u;
        return Storage<S>::from_f_sr(v * k.isw[a], r);
    } else {
        return S(v);
    }
}

// fp64 sum of the wall terms in a fixed order: term k goes to accumulator
// k mod 4, the four are combined as (a0 + a1) + (a2 + a3).  Four interleaved
// chains instead of one keep the fp64 latency of a wall node short; every
// kernel uses this order, so all paths give the same bits.
struct Acc4 {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    __device__ __forceinline__ void add(int k, double v) {
        switch (k & 3) {
            case 0: a0 += v; break;
            case 1: a1 += v; break;
            case 2: a2 += v; break;
            default: a3 += v; break;
        }
    }
    __device__ __forceinline__ double sum() const { return (a0 + a1) + (a2 + a3); }
};

// Wall flux balance (Eq. nm.15) for landing column x, in deviation form:
// returns dPsi = sum_out d_b / sum_in |e_y| w  so that an unknown incoming
// population is d_a = dPsi * w_a, i.e. fbar_a = Psi rho_w w_a (Eq. nm.14).
// Outgoing populations b (e_y < 0 at the bottom wall, e_y > 0 at the top)
// cross the wall from their |e_y| rows nearest to it and are credited to the
// column they land on, so the source column is x - e_x.  Terms in plane order,
// nearest row first; fp64 accumulation (Acc4) in every precision; the fill
// d_a = dPsi w_a is formed in the compute type.
template <typename S, typename C, class LD>
__device__ __forceinline__ double wall_dpsi_by(const KParams<C>& k, int x, bool bottom,
                                               const LD& ld) {
    Acc4 acc;
    int t = 0;
    for (int b = k.R; b < k.V; ++b) {
        const int ey = k.ey[b];
        if (bottom ? (ey >= 0) : (ey <= 0)) continue;
        int xs = x - k.sx[b];
        xs += (xs < 0) ? k.Nx : 0;
        const int n = bottom ? -ey : ey;
        for (int j = 0; j < n; ++j) {
            const int row = bottom ? j : (k.Ny - 1 - j);
            acc.add(t++, (double)ld_pop<S, C>(k, ld(b, row, xs), b));
        }
    }
    return acc.sum() * k.inv_den;
}

// The same sum read from a lattice in global memory ([V][Ny][Nx] planes).
template <typename S, typename C>
__device__ __noinline__ double wall_dpsi(const KParams<C>& k, const S* __restrict__ src, int x,
                                         bool bottom) {
    return wall_dpsi_by<S, C>(k, x, bottom, [&](int b, int row, int xs) {
        return src[(long long)b * k.plane + (long long)row * k.Nx + xs];
    });
}

// The same sum spread over the first four lanes of a node (lane p of the node,
// `lead` the node's first lane; every lane of the warp calls this): lane j < 4
// of a node with `mine` set adds the terms j, j + 4, ... -- accumulator j of
// Acc4 -- and two shuffles form (a0 + a1) + (a2 + a3) on the first lane, whose
// result every lane of the node receives: the bits of wall_dpsi_by.
template <typename S, typename C, class LD>
__device__ __forceinline__ double wall_dpsi_lanes(const KParams<C>& k, int x, bool bottom,
                                                  bool mine, int p, int lead, const LD& ld) {
    constexpr unsigned FULL = 0xffffffffu;
    double acc = 0.0;
    if (mine && p < 4) {
        int t = 0;
        for (int b = k.R; b < k.V; ++b) {
            const int ey = k.ey[b];
            if (bottom ? (ey >= 0) : (ey <= 0)) continue;
            int xs = x - k.sx[b];
            xs += (xs < 0) ? k.Nx : 0;
            const int n = bottom ? -ey : ey;
            for (int j = 0; j < n; ++j, ++t) {
                if ((t & 3) != p) continue;
                const int row = bottom ? j : (k.Ny - 1 - j);
                acc += (double)ld_pop<S, C>(k, ld(b, row, xs), b);
            }
        }
    }
    const int lane = threadIdx.x & 31;
    const double s2 = acc + __shfl_sync(FULL, acc, (lane + 1) & 31);
    const double tot = s2 + __shfl_sync(FULL, s2, (lane + 2) & 31);
    return __shfl_sync(FULL, tot * k.inv_den, lead);
}

// Number of wall terms of the planes before plane a of a compiled set.
template <class SET, bool BOTTOM>
__host__ __device__ constexpr int wall_terms_before(int a) {
    int t = 0;
    for (int b = 0; b < a; ++b) {
        const int ey = b < SET::R ? 0 : (b < SET::R + SET::P ? SET::ey[b - SET::R] : -SET::ey[b - SET::R - SET::P]);
        if (BOTTOM ? ey < 0 : ey > 0) t += BOTTOM ? -ey : ey;
    }
    return t;
}

// The same sum for a compiled set, unrolled: term(plane, j) gives the
// outgoing population of plane `plane` (an integral_constant) that crossed
// from the j-th row off the wall.
template <class SET, bool BOTTOM, int A, class TERM>
__device__ __forceinline__ void wall_add_plane(Acc4& acc, const TERM& term) {
    constexpr int ey = A < SET::R ? 0 : (A < SET::R + SET::P ? SET::ey[A - SET::R] : -SET::ey[A - SET::R - SET::P]);
    if constexpr (BOTTOM ? ey < 0 : ey > 0) {
        constexpr int n = BOTTOM ? -ey : ey;
        constexpr int t0 = wall_terms_before<SET, BOTTOM>(A);
#pragma unroll
        for (int j = 0; j < n; ++j) acc.add(t0 + j, term(std::integral_constant<int, A>{}, j));
    }
}

template <class SET, bool BOTTOM, class TERM, int... I>
__device__ __forceinline__ double wall_sum_ct(const TERM& term, std::integer_sequence<int, I...>) {
    Acc4 acc;
    (wall_add_plane<SET, BOTTOM, I>(acc, term), ...);
    return acc.sum();
}

// Wall balance of a compiled set on a lattice in device memory.
template <class SET, typename S, typename C, bool BOTTOM>
__device__ __forceinline__ double wall_dpsi_ct(const KParams<C>& k, const S* __restrict__ src, int x) {
    constexpr int V = SET::R + 2 * SET::P;
    auto term = [&](auto bc, int j) {
        constexpr int b = decltype(bc)::value;
        int xs = x - k.sx[b];
        xs += (xs < 0) ? k.Nx : 0;
        const int row = BOTTOM ? j : (k.Ny - 1 - j);
        return (double)ld_pop<S, C>(k, src[(long long)b * k.plane + (long long)row * k.Nx + xs], b);
    };
    return wall_sum_ct<SET, BOTTOM>(term, std::make_integer_sequence<int, V>{}) * k.inv_den;
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
    // compile-time-velocity path, g along x (g.xi = c g_x e_x):
    C trcg;                   // tau rho c g_x:  even part += e_x trcg s
    C k0, cqxx, cqxy, cqyy;   // odd part += e_x (k0 + cqxx ex^2 + cqxy 2 ex ey + cqyy ey^2)
};

template <int N, typename C>
__device__ __forceinline__ CellCoef<C> cell_coef(const KParams<C>& k, C drho, C Jx, C Jy,
                                                 C Kxx, C Kxy, C Kyy) {
    CellCoef<C> q;
    q.drho = drho;
    q.rho = C(1) + drho;
    const C inv = C(1) / q.rho;
    // Eq. nm.10: rho u = sum fbar xi + (dt/2) rho g
    q.ux = fma(mul_rn(k.c, Jx), inv, k.hdt_gx);
    q.uy = fma(mul_rn(k.c, Jy), inv, k.hdt_gy);
    q.utx = mul_rn(k.c, q.ux);
    q.uty = mul_rn(k.c, q.uy);
    const C u2 = fma(q.ux, q.ux, mul_rn(q.uy, q.uy));
    // f0/(rho w) - 1 of Eq. nm.3 (+ the N = 4 Hermite term of Eq. equi.hermite)
    // with s = u.xi, t = s^2:
    //   even: (t - u2)/2 + [N>=4] (t^2 - 6 t u2 + 3 u2^2)/24
    //   odd:  s + [N>=3] s (t - 3 u2)/6
    // (products with powers of two are exact)
    q.a0 = fma(q.rho, N >= 4 ? fma(C(0.125) * u2, u2, C(-0.5) * u2) : C(-0.5) * u2, drho);
    q.a1 = mul_rn(q.rho, C(0.5) - (N >= 4 ? C(0.25) * u2 : C(0)));
    q.a2 = N >= 4 ? mul_rn(q.rho, C(1.0 / 24.0)) : C(0);
    q.b0 = N >= 3 ? mul_rn(q.rho, C(1) - C(0.5) * u2) : q.rho;
    q.b1 = N >= 3 ? mul_rn(q.rho, C(1.0 / 6.0)) : C(0);
    q.tr = mul_rn(k.tau, q.rho);
    if (k.force) {
        // even force part of Eq. nm.4: tau rho ((g.xi)(u.xi) - u.g)
        q.a0 = fma(-q.tr, fma(q.ux, k.gx, mul_rn(q.uy, k.gy)), q.a0);
        // A = Pi - rho delta, Pi the momentum flux of f = (2 tau fbar + dt feq)
        // / (2 tau + dt) (Eq. nm.7 inverted), Pibar = delta + c^2 K and
        // Pi_eq = rho (delta + u u + tau (g u + u g)) (exact for Q >= N + 2):
        //   (2 tau + dt) A = -2 tau drho delta + 2 tau c^2 K
        //                    + dt rho (u u + tau (g u + u g))
        const C tdr = mul_rn(k.dt, q.rho);
        const C tgx = k.tgx, tgy = k.tgy;
        const C Axx = mul_rn(fma(k.two_tau, fma(k.c2, Kxx, -drho),
                                 mul_rn(tdr, fma(q.ux, q.ux, mul_rn(tgx, q.ux)))), k.inv_2tau_dt);
        const C Ayy = mul_rn(fma(k.two_tau, fma(k.c2, Kyy, -drho),
                                 mul_rn(tdr, fma(q.uy, q.uy, mul_rn(tgy, q.uy)))), k.inv_2tau_dt);
        const C Axy = mul_rn(fma(k.ttc2, Kxy,
                                 mul_rn(tdr, fma(q.ux, q.uy, mul_rn(k.tau, fma(k.gx, q.uy,
                                                                              mul_rn(k.gy, q.ux)))))),
                             k.inv_2tau_dt);
        if (N >= 3) {
            // third-order force term (1/2) A:((g.xi) H2(xi) - 2 g xi)
            const C htc2 = k.htc2, tc = k.tc;
            q.qxx = mul_rn(htc2, Axx);
            q.qxy = mul_rn(htc2, Axy);   // multiplies 2 ex ey
            q.qyy = mul_rn(htc2, Ayy);
            q.qtr = mul_rn(k.half_tau, Axx + Ayy);
            q.hx = mul_rn(tc, fma(k.gx, Axx, mul_rn(k.gy, Axy)));
            q.hy = mul_rn(tc, fma(k.gx, Axy, mul_rn(k.gy, Ayy)));
        } else {
            q.qxx = q.qxy = q.qyy = q.qtr = q.hx = q.hy = C(0);
        }
        const C cg = k.cg;
        q.trcg = mul_rn(q.tr, cg);
        q.k0 = mul_rn(cg, q.tr - q.qtr);
        q.cqxx = mul_rn(cg, q.qxx);
        q.cqxy = mul_rn(cg, q.qxy);
        q.cqyy = mul_rn(cg, q.qyy);
    }
    return q;
}

// Constants of the +-e pair p (positive member e = (ex, ey)).
template <typename C>
struct PairConst {
    C ex, ey, exx, exy2, eyy, ge, omw;
};

template <typename C>
__device__ __forceinline__ PairConst<C> pair_const(const KParams<C>& k, int p) {
    return PairConst<C>{k.pex[p], k.pey[p], k.pexx[p], k.pexy2[p], k.peyy[p], k.pge[p], k.pomw[p]};
}

// Relax one +-e pair (planes fp, fm) in place:
//   d* = (1 - omega) d + omega w (feq/w - 1),  feq/w - 1 = Ge +- Go.
template <bool FORCE, typename C>
__device__ __forceinline__ void pair_update_pc(const KParams<C>& k, const CellCoef<C>& q,
                                               const PairConst<C>& pc, C& fp, C& fm) {
    const C ex = pc.ex, ey = pc.ey;
    const C s = fma(q.uty, ey, q.utx * ex);
    const C t = mul_rn(s, s);
    C Ge = fma(t, fma(t, q.a2, q.a1), q.a0);
    C Go = mul_rn(s, fma(t, q.b1, q.b0));
    if (FORCE) {
        const C ge = pc.ge;
        // odd force part: tau rho (g.xi) + (tau/2)((g.xi) Q - 2 (g.A).xi)
        const C halfQ = fma(q.qxx, pc.exx, fma(q.qxy, pc.exy2, fma(q.qyy, pc.eyy, -q.qtr)));
        Ge = fma(mul_rn(q.tr, ge), s, Ge);
        Go = fma(ge, q.tr + halfQ, Go) - fma(q.hx, ex, q.hy * ey);
    }
    const C X = mul_rn(pc.omw, Ge);
    fp = fma(k.one_m_omega, fp, fma(pc.omw, Go, X));
    fm = fma(k.one_m_omega, fm, fma(-pc.omw, Go, X));
}

template <bool FORCE, typename C>
__device__ __forceinline__ void pair_update(const KParams<C>& k, const CellCoef<C>& q, int p,
                                            C& fp, C& fm) {
    pair_update_pc<FORCE, C>(k, q, pair_const(k, p), fp, fm);
}

// Flag a density that is not in (0, inf) (negative, zero, infinite or NaN).
// Tested on the bit pattern: as a signed integer a positive finite non-zero
// value lies strictly between 0 and the pattern of +inf; the integer compares
// keep the test off the (slow) fp64 pipe.
template <typename C>
__device__ __forceinline__ void flag_density(const CellCoef<C>& q, unsigned int* status) {
    bool ok;
    if constexpr (sizeof(C) == 8) {
        const long long bits = __double_as_longlong(q.rho);
        ok = bits > 0 && bits < 0x7ff0000000000000ll;
    } else {
        const int bits = __float_as_int(q.rho);
        ok = bits > 0 && bits < 0x7f800000;
    }
    if (!ok) atomicOr(status, 1u);
}

template <typename C>
__device__ __forceinline__ void store_moments(const CellCoef<C>& q, int cell, const DevBufs& b) {
    b.rho[cell] = 1.0 + (double)q.drho;
    b.ux[cell] = (double)q.ux;
    b.uy[cell] = (double)q.uy;
}

template <typename C>
__device__ __forceinline__ void emit_moments(const KParams<C>& k, const CellCoef<C>& q, int cell,
                                             const DevBufs& b) {
    if (k.emit) store_moments<C>(q, cell, b);
}

// Pull one population of plane a into node (x, y) of an interior row.
template <typename S, typename C>
__device__ __forceinline__ C pull(const KParams<C>& k, const S* __restrict__ src, int a, int x, int y) {
    int xs = x - k.sx[a];
    xs += (xs < 0) ? k.Nx : 0;
    return ld_pop<S, C>(k, src[(long long)a * k.plane + (long long)(y - k.ey[a]) * k.Nx + xs], a);
}

// Populations of a wall node of a compiled set: the fill for those whose
// source lies beyond a wall, the pull for the others.
template <class SET, typename S, typename C, int A>
__device__ __forceinline__ C wall_value(const KParams<C>& k, const S* __restrict__ src, int x, int y,
                                        C pb, C pt) {
    constexpr int EY = A < SET::R ? 0 : (A < SET::R + SET::P ? SET::ey[A - SET::R] : -SET::ey[A - SET::R - SET::P]);
    const int ys = y - EY;
    if (ys < 0) return pb * k.cw[A];
    if (ys >= k.Ny) return pt * k.cw[A];
    return pull<S, C>(k, src, A, x, y);
}

template <class SET, typename S, typename C, int... I>
__device__ __forceinline__ void pull_wall_ct(const KParams<C>& k, const S* __restrict__ src, int x,
                                             int y, C* f, std::integer_sequence<int, I...>) {
    const C pb = y < k.maxey ? C(wall_dpsi_ct<SET, S, C, true>(k, src, x)) : C(0);
    const C pt = y >= k.Ny - k.maxey ? C(wall_dpsi_ct<SET, S, C, false>(k, src, x)) : C(0);
    ((f[I] = wall_value<SET, S, C, I>(k, src, x, y, pb, pt)), ...);
}

// ---- compile-time velocity sets ---------------------------------------------
// With e known at compile time, products with e components 0 and +-1 vanish
// or become additions (IEEE rules forbid the compiler from folding x * 0).

template <int E, typename C>
__device__ __forceinline__ C mulc(C v) {          // E v, E != 0
    if constexpr (E == 1) return v;
    else if constexpr (E == -1) return -v;
    else return mul_rn(C(E), v);
}

template <int E, typename C>
__device__ __forceinline__ C fmac(C a, C v) {     // a + E v
    if constexpr (E == 0) return a;
    else if constexpr (E == 1) return a + v;
    else if constexpr (E == -1) return a - v;
    else return fma(C(E), v, a);
}

template <int EX, int EY, typename C>
__device__ __forceinline__ C lin(C x, C y) {      // EX x + EY y, (EX, EY) != 0
    if constexpr (EX == 0) return mulc<EY>(y);
    else if constexpr (EY == 0) return mulc<EX>(x);
    else return fmac<EY>(mulc<EX>(x), y);
}

template <int EX, int EY, typename C>
__device__ __forceinline__ void moment_pair(C fp, C fm, C& drho, C& Jx, C& Jy, C& Kxx, C& Kxy,
                                            C& Kyy) {
    const C sum = fp + fm, dif = fp - fm;
    drho += sum;
    Jx = fmac<EX>(Jx, dif);
    Jy = fmac<EY>(Jy, dif);
    Kxx = fmac<EX * EX>(Kxx, sum);
    Kxy = fmac<EX * EY>(Kxy, sum);
    Kyy = fmac<EY * EY>(Kyy, sum);
}

// Relax the pair (+e, -e), e = (EX, EY) known at compile time; same
// arithmetic as pair_update with the force along x.
template <int EX, int EY, int N, bool FORCE, typename C>
__device__ __forceinline__ void pair_update_ct(const CellCoef<C>& q, C omw, C omo, C& fp, C& fm) {
    const C s = lin<EX, EY>(q.utx, q.uty);
    const C t = mul_rn(s, s);
    C Ge = N >= 4 ? fma(t, fma(t, q.a2, q.a1), q.a0) : fma(t, q.a1, q.a0);
    C Go = N >= 3 ? mul_rn(s, fma(t, q.b1, q.b0)) : mul_rn(s, q.b0);
    if constexpr (FORCE) {
        if constexpr (EX != 0) {
            // even: tau rho (g.xi) s; odd: (g.xi)(tau rho + (tau/2) Q)
            Ge = fma(mulc<EX>(q.trcg), s, Ge);
            C inner = q.k0;
            inner = fmac<EX * EX>(inner, q.cqxx);
            inner = fmac<2 * EX * EY>(inner, q.cqxy);
            inner = fmac<EY * EY>(inner, q.cqyy);
            Go = fmac<EX>(Go, inner);
        }
        Go = Go - lin<EX, EY>(q.hx, q.hy);      // - tau (g.A).xi
    }
    const C X = mul_rn(omw, Ge);
    fp = fma(omo, fp, fma(omw, Go, X));
    fm = fma(omo, fm, fma(-omw, Go, X));
}

template <class SET, typename C, int... I>
__device__ __forceinline__ void moments_ct(const C* f, C& drho, C& Jx, C& Jy, C& Kxx, C& Kxy,
                                           C& Kyy, std::integer_sequence<int, I...>) {
    (moment_pair<SET::ex[I], SET::ey[I], C>(f[SET::R + I], f[SET::R + SET::P + I], drho, Jx, Jy,
                                            Kxx, Kxy, Kyy), ...);
}

template <class SET, int N, bool FORCE, typename C, int... I>
__device__ __forceinline__ void relax_ct(const KParams<C>& k, const CellCoef<C>& q, C* f,
                                         std::integer_sequence<int, I...>) {
    (pair_update_ct<SET::ex[I], SET::ey[I], N, FORCE, C>(q, k.pomw[I], k.one_m_omega,
                                                         f[SET::R + I], f[SET::R + SET::P + I]), ...);
}

// Middle path of a tile whose rows all lie at least max|e_y| rows from both
// walls (the nodes may wrap around x): the source of plane a is
// cell - off[a] + dx[a] (+ Nx when x - e_x wraps below 0), with
// sp[a] = lattice + a plane - off[a].
template <int V, typename S, typename C, typename PTR>
__device__ __forceinline__ void pull_rows(const KParams<C>& k, const PTR& sp, int cell, C* f) {
    const int y = cell / k.Nx;
    const int x = cell - y * k.Nx;
#pragma unroll
    for (int a = 0; a < V; ++a) {
        const int i = cell + k.dx[a] + (x < k.sx[a] ? k.Nx : 0);
        f[a] = ld_pop<S, C>(k, static_cast<const S*>(sp[a])[i], a);
    }
}

// e_x of plane a of a compiled set (rest, the P pair members, their negatives)
template <class SET>
__host__ __device__ constexpr int plane_ex(int a) {
    return a < SET::R ? 0 : (a < SET::R + SET::P ? SET::ex[a - SET::R] : -SET::ex[a - SET::R - SET::P]);
}

// Rows path with e_x known at compile time (all rows of the node away from the
// walls).  sp[a] = lattice + a plane - (e_y Nx + e_x) (a pointer, or for the
// single-solve kernel a byte address).  With Nx >= max|e_x|
// the x wrap is one compare against a constant; with Nx = 1 every source lies
// in the same column and the pull is cell + e_x.
template <class SET, typename S, typename C, int A, class PTR>
__device__ __forceinline__ C pull_col(const KParams<C>& k, const PTR& sp, int cell, int x,
                                      int Nx) {
    constexpr int EX = plane_ex<SET>(A);
    int i;
    if constexpr (EX == 0) {
        i = cell;
    } else if constexpr (EX > 0) {
        i = cell + (x < EX ? Nx : 0);
    } else {
        i = cell + (x < Nx + EX ? 0 : -Nx);
    }
    return ld_pop<S, C>(k, ld_stream(static_cast<const S*>(sp[A]) + i), A);
}

template <class SET, typename S, typename C, int A, class PTR>
__device__ __forceinline__ C pull_col1(const KParams<C>& k, const PTR& sp, int cell) {
    return ld_pop<S, C>(k, ld_stream(static_cast<const S*>(sp[A]) + cell + plane_ex<SET>(A)), A);
}

template <class SET, typename S, typename C, class PTR, int... I>
__device__ __forceinline__ void pull_rows_ct(const KParams<C>& k, const PTR& sp, int cell,
                                             C* f, std::integer_sequence<int, I...>) {
    const int Nx = k.Nx;
    if (Nx == 1) {
        ((f[I] = pull_col1<SET, S, C, I, PTR>(k, sp, cell)), ...);
    } else {
        const int x = cell % Nx;
        ((f[I] = pull_col<SET, S, C, I, PTR>(k, sp, cell, x, Nx)), ...);
    }
}

// Rows-path pull of a compiled set: the compile-time forms where they apply.
template <class SET, typename S, typename C, class PTR>
__device__ __forceinline__ void pull_rows_any(const KParams<C>& k, const PTR& sp, int cell, C* f) {
    constexpr int V = SET::R + 2 * SET::P;
    if (k.Nx == 1 || k.Nx >= k.maxex)
        pull_rows_ct<SET, S, C>(k, sp, cell, f, std::make_integer_sequence<int, V>{});
    else
        pull_rows<V, S, C>(k, sp, cell, f);
}

// Fused step for a compiled velocity set: the V populations stay in registers
// between the moment pass and the relaxation pass.
//  - fast path (block-uniform): the block's nodes lie in one row at least
//    max|e_y| rows from both walls and max|e_x| columns from both ends, so
//    every pull is a fixed offset from the node: one address per population;
//  - rows path (block-uniform): all rows of the block are away from the walls
//    but nodes may wrap around x (narrow channels, x ends): a compare and a
//    select per population;
//  - general path: periodic wrap in x and the diffuse-wall fill near walls.
template <class SET, int N, typename S, typename C>
__global__ void __launch_bounds__(kBlock, min_blocks_for(SET::R + 2 * SET::P, sizeof(C)))
k_step_ct(const __grid_constant__ KParams<C> k, const S* __restrict__ src, S* __restrict__ dst,
          const DevBufs b) {
    constexpr int R = SET::R, P = SET::P, V = R + 2 * P;
    const int c0 = blockIdx.x * kBlock;
    const int cell = c0 + threadIdx.x;
    const int y0 = c0 / k.Nx;
    const int x0 = c0 - y0 * k.Nx;
    const bool fast = x0 >= k.maxex && x0 + kBlock - 1 + k.maxex < k.Nx && y0 >= k.maxey &&
                      y0 < k.Ny - k.maxey;
    const int y1 = (min(c0 + kBlock, k.ncell) - 1) / k.Nx;
    const bool rows = !fast && y0 >= k.maxey && y1 < k.Ny - k.maxey;
    C f[V];
    if (fast) {
#pragma unroll
        for (int a = 0; a < V; ++a) f[a] = ld_pop<S, C>(k, ld_stream(static_cast<const S*>(k.srcf[a]) + cell), a);
    } else if (rows) {
        if (cell >= k.ncell) return;
        pull_rows_any<SET, S, C>(k, k.srcf, cell, f);
    } else {
        if (cell >= k.ncell) return;
        const int y = cell / k.Nx;
        const int x = cell - y * k.Nx;
        const bool nb = y < k.maxey, nt = y >= k.Ny - k.maxey;
        if (!nb && !nt)            // a node away from the walls in a tile that touches one
            pull_rows_any<SET, S, C>(k, k.srcf, cell, f);
        else
            pull_wall_ct<SET, S, C>(k, src, x, y, f, std::make_integer_sequence<int, V>{});
    }
    C drho = R ? f[0] : C(0), Jx = 0, Jy = 0, Kxx = 0, Kxy = 0, Kyy = 0;
    moments_ct<SET, C>(f, drho, Jx, Jy, Kxx, Kxy, Kyy, std::make_integer_sequence<int, P>{});
    const CellCoef<C> q = cell_coef<N, C>(k, drho, Jx, Jy, Kxx, Kxy, Kyy);
    if (R) f[0] = fma(k.one_m_omega, f[0], k.omw_rest * q.a0);
    if (k.force)
        relax_ct<SET, N, true, C>(k, q, f, std::make_integer_sequence<int, P>{});
    else
        relax_ct<SET, N, false, C>(k, q, f, std::make_integer_sequence<int, P>{});
    unsigned rs = sr_seed<S, C>(k.seed, cell);
#pragma unroll
    for (int a = 0; a < V; ++a) static_cast<S*>(k.dstp[a])[cell] = st_pop<S, C>(k, f[a], a, rs);
    emit_moments<C>(k, q, cell, b);
    flag_density<C>(q, b.status);
}

// Sum six per-lane values over the LP lanes of a node (LP = 8, 16, 32; lane p
// of the node), leaving the six sums on every lane.  The summation tree is the
// butterfly's -- partners p ^ LP/2, p ^ LP/4, ..., p ^ 1, each sum formed as
// a + b of the two partners' values -- but the first three levels are a
// reduce-scatter over eight slots (the six values and two zeros): at each
// level a lane keeps half of its slots and adds the partner's copy of them, so
// the level costs 4, 2, 1 additions instead of 6.  A lane then holds slot
// (p / (LP/8)) mod 8; the last levels add that one value, and shuffles gather
// the six sums.  IEEE addition is commutative, so every sum has the bits of the
// six-wide butterfly.
template <int LP, typename C>
__device__ __forceinline__ void node_sum6(C (&m)[6], int p) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int B1 = LP / 2, B2 = LP / 4, B3 = LP / 8;
    C v4[4];
    {   // level 1: keep slots 0-3 (bit clear) or 4-7 (bit set), send the others
        const bool hi = (p & B1) != 0;
        const C s8[8] = {m[0], m[1], m[2], m[3], m[4], m[5], C(0), C(0)};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const C keep = hi ? s8[4 + i] : s8[i];
            const C send = hi ? s8[i] : s8[4 + i];
            v4[i] = keep + __shfl_xor_sync(FULL, send, B1);
        }
    }
    C v2[2];
    {
        const bool hi = (p & B2) != 0;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const C keep = hi ? v4[2 + i] : v4[i];
            const C send = hi ? v4[i] : v4[2 + i];
            v2[i] = keep + __shfl_xor_sync(FULL, send, B2);
        }
    }
    C v;
    {
        const bool hi = (p & B3) != 0;
        const C keep = hi ? v2[1] : v2[0];
        const C send = hi ? v2[0] : v2[1];
        v = keep + __shfl_xor_sync(FULL, send, B3);
    }
#pragma unroll
    for (int o = B3 / 2; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    const int lead = (threadIdx.x & 31) - p;
#pragma unroll
    for (int i = 0; i < 6; ++i) m[i] = __shfl_sync(FULL, v, lead + i * B3);
}

// One node of the tiny-channel step on LP lanes (a power of 2 >= P): lane p of
// the node holds the pair (R + p, R + P + p) with constants pc and streamed (or
// wall-filled) values fp, fm (0 on lanes p >= P), lane 0 also the rest value
// f0 (0 without a rest velocity).  The moments are summed over the node's
// lanes by butterfly shuffles and every lane derives the node's coefficients;
// put(a, v) stores the post-collision population a.  The shuffles span the
// warp: every lane of the warp calls this, `node` false on lanes without one.
template <int LP, int N, typename C, class PUT>
__device__ __forceinline__ CellCoef<C> warp_node(const KParams<C>& k, int p, bool node,
                                                 const PairConst<C>& pc, C fp, C fm, C f0,
                                                 const PUT& put) {
    const bool act = node && p < k.P;
    const C sum = fp + fm, dif = fp - fm;
    C m[6] = {sum + f0, act ? mul_rn(pc.ex, dif) : C(0), act ? mul_rn(pc.ey, dif) : C(0),
              act ? mul_rn(pc.exx, sum) : C(0), act ? mul_rn(pc.exy2, sum) : C(0),
              act ? mul_rn(pc.eyy, sum) : C(0)};
    node_sum6<LP, C>(m, p);
    CellCoef<C> q{};
    if (!node) return q;
    q = cell_coef<N, C>(k, m[0], m[1], m[2], m[3], C(0.5) * m[4], m[5]);
    if (act) {
        if (k.force)
            pair_update_pc<true, C>(k, q, pc, fp, fm);
        else
            pair_update_pc<false, C>(k, q, pc, fp, fm);
        put(k.R + p, fp);
        put(k.R + k.P + p, fm);
    }
    if (p == 0 && k.R) put(0, fma(k.one_m_omega, f0, k.omw_rest * q.a0));
    return q;
}

// Step for tiny channels: warp_node on every node, one warp per block, so a
// channel of a few hundred nodes spreads over many SMs instead of running on
// one (the fp64 step of a 64-node channel is otherwise bound by a single SM's
// fp64 lanes).
template <int LP, int N, typename S, typename C>
__global__ void __launch_bounds__(32)
k_step_warp(const __grid_constant__ KParams<C> k, const S* __restrict__ src, S* __restrict__ dst,
            const DevBufs b) {
    constexpr int G = 32 / LP;                 // nodes per warp
    const int lane = threadIdx.x;
    const int cell = blockIdx.x * G + lane / LP;
    const int p = lane % LP;
    const bool node = cell < k.ncell;
    int y = 0, x = 0;
    if (node) {
        y = cell / k.Nx;
        x = cell - y * k.Nx;
    }
    const bool wb = node && y < k.maxey, wt = node && y >= k.Ny - k.maxey;
    auto ld = [&](int b, int row, int xs) {
        return src[(long long)b * k.plane + (long long)row * k.Nx + xs];
    };
    const int lead = lane - p;
    const C pb = __any_sync(0xffffffffu, wb) ? C(wall_dpsi_lanes<S, C>(k, x, true, wb, p, lead, ld))
                                             : C(0);
    const C pt = __any_sync(0xffffffffu, wt) ? C(wall_dpsi_lanes<S, C>(k, x, false, wt, p, lead, ld))
                                             : C(0);
    auto value = [&](int a) -> C {
        const int ys = y - k.ey[a];
        if (ys < 0) return mul_rn(pb, k.cw[a]);
        if (ys >= k.Ny) return mul_rn(pt, k.cw[a]);
        return pull<S, C>(k, src, a, x, y);
    };
    const bool act = node && p < k.P;
    const PairConst<C> pc = pair_const(k, act ? p : 0);
    const C fp = act ? value(k.R + p) : C(0);
    const C fm = act ? value(k.R + k.P + p) : C(0);
    const C f0 = (node && p == 0 && k.R) ? value(0) : C(0);
    unsigned rs = sr_seed<S, C>(k.seed, cell);
    auto put = [&](int a, C v) { dst[(long long)a * k.plane + cell] = st_pop<S, C>(k, v, a, rs); };
    const CellCoef<C> q = warp_node<LP, N, C>(k, p, node, pc, fp, fm, f0, put);
    if (node && p == 0) {
        emit_moments<C>(k, q, cell, b);
        flag_density<C>(q, b.status);
    }
}

template <int N, typename S, typename C>
cudaError_t launch_warp(const KParams<C>& k, int LP, const S* src, S* dst, const DevBufs& b,
                        cudaStream_t st) {
    const int G = 32 / LP;
    const dim3 g((k.ncell + G - 1) / G);
    switch (LP) {
        case 8: k_step_warp<8, N, S, C><<<g, 32, 0, st>>>(k, src, dst, b); break;
        case 16: k_step_warp<16, N, S, C><<<g, 32, 0, st>>>(k, src, dst, b); break;
        default: k_step_warp<32, N, S, C><<<g, 32, 0, st>>>(k, src, dst, b); break;
    }
    return cudaGetLastError();
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
    C pb = C(0), pt = C(0);
    double r0 = 0.0;
    if (INIT) {
        r0 = rho0[cell] - 1.0;
    } else {
        if (y < k.maxey) pb = C(wall_dpsi<S, C>(k, src, x, true));
        if (y >= k.Ny - k.maxey) pt = C(wall_dpsi<S, C>(k, src, x, false));
    }
    auto value = [&](int a) -> C {
        if (INIT) return C(r0 * k.w[a]);
        const int ys = y - k.ey[a];
        if (ys < 0) return pb * k.cw[a];
        if (ys >= k.Ny) return pt * k.cw[a];
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
    unsigned rs = sr_seed<S, C>(k.seed, cell);
    if (R) dst[cell] = st_pop<S, C>(k, fma(k.one_m_omega, value(0), k.omw_rest * q.a0), 0, rs);
    for (int p = 0; p < P; ++p) {
        C fp = value(R + p), fm = value(R + P + p);
        if (k.force)
            pair_update<true, C>(k, q, p, fp, fm);
        else
            pair_update<false, C>(k, q, p, fp, fm);
        dst[(long long)(R + p) * k.plane + cell] = st_pop<S, C>(k, fp, R + p, rs);
        dst[(long long)(R + P + p) * k.plane + cell] = st_pop<S, C>(k, fm, R + P + p, rs);
    }
    emit_moments<C>(k, q, cell, b);
    flag_density<C>(q, b.status);
}

// Launch helpers -------------------------------------------------------------

template <typename C>
inline dim3 grid_for(const KParams<C>& k) { return dim3((k.ncell + kBlock - 1) / kBlock); }

// Dispatch: a compiled velocity set (dvm_sets.h) gets its register-resident
// kernel, any other DVM the generic kernel.
template <int N, typename S, typename C>
cudaError_t launch_step_n(const KParams<C>& k, const S* src, S* dst, const DevBufs& b,
                          cudaStream_t st) {
    const dim3 g = grid_for(k);
    // fp64 and fp32 channels too small to fill the GPU with one node per
    // thread: several lanes per node (k_step_warp) spread the work over more
    // SMs, and the same body runs resident chunks on a cluster (k_cluster.cu)
    if (sizeof(C) == 8 || sizeof(S) == 4) {
        const int LP = warp_path_lanes(k.P, k.ncell);
        if (LP) return launch_warp<N, S, C>(k, LP, src, dst, b, st);
    }
    switch (k.set_id) {
        case 0: k_step_ct<SetD2V16, N, S, C><<<g, kBlock, 0, st>>>(k, src, dst, b); break;
        case 1: k_step_ct<SetD2V32, N, S, C><<<g, kBlock, 0, st>>>(k, src, dst, b); break;
        case 2: k_step_ct<SetD2V33, N, S, C><<<g, kBlock, 0, st>>>(k, src, dst, b); break;
        case 3: k_step_ct<SetD2V53, N, S, C><<<g, kBlock, 0, st>>>(k, src, dst, b); break;
        case 4: k_step_ct<SetD2V40, N, S, C><<<g, kBlock, 0, st>>>(k, src, dst, b); break;
        case 5: k_step_ct<SetD2V48, N, S, C><<<g, kBlock, 0, st>>>(k, src, dst, b); break;
        default: k_generic<N, false, S, C><<<g, kBlock, 0, st>>>(k, src, nullptr, dst, b);
    }
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
