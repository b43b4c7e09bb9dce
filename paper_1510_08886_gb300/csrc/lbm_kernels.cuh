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
//
// The compiled-set kernels round two values at once with the hardware's
// stochastically rounding conversion (cvt.rs, random bits supplied by the
// caller): a in the upper half of the result, b in the lower half.
template <> struct Storage<__half> {
    static constexpr bool scaled = true;
    static __device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half from_f(float v) { return __float2half_rn(v); }
    // fp32 keeps 13 more mantissa bits than fp16
    static __device__ __forceinline__ __half from_f_sr(float v, unsigned r) {
        return __float2half_rz(__uint_as_float(__float_as_uint(v) + (r >> 19)));
    }
    static __device__ __forceinline__ void sr2(float a, float b, unsigned r, __half& ha, __half& hb) {
        unsigned d;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(a), "f"(b), "r"(r));
        ha = __ushort_as_half((unsigned short)(d >> 16));
        hb = __ushort_as_half((unsigned short)(d & 0xffffu));
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
    static __device__ __forceinline__ void sr2(float a, float b, unsigned r, __nv_bfloat16& ha,
                                               __nv_bfloat16& hb) {
        unsigned d;
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(a), "f"(b), "r"(r));
        ha = __ushort_as_bfloat16((unsigned short)(d >> 16));
        hb = __ushort_as_bfloat16((unsigned short)(d & 0xffffu));
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
// on the 4096 x 512 fp32 step).
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
__device__ __forceinline__ S ld_stream(const S* p) {      // 16-bit planes: plain load
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

// Register value of a stored population in the compiled-set kernels: the
// deviation d itself for fp64/fp32 storage, h = d / (w_a S) for the 16-bit
// formats (their moment sums weigh h with w_a S, their relaxation works in h).
template <typename S, typename C>
__device__ __forceinline__ C ld_val(S v) {
    if constexpr (Storage<S>::scaled) return Storage<S>::to_f(v);
    else return C(v);
}

// Wall fill d_a = dPsi w_a in register units (dPsi / S for 16-bit storage).
template <typename S, typename C>
__device__ __forceinline__ C fill_val(const KParams<C>& k, C dpsi, int a) {
    if constexpr (Storage<S>::scaled) return mul_rn(dpsi, k.fill_h);
    else return mul_rn(dpsi, k.cw[a]);
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

// emit 1: write the fp64 moments of this step; emit 2: add them to the
// fields (time averages, lbm_average)
template <typename C>
__device__ __forceinline__ void emit_moments(const KParams<C>& k, const CellCoef<C>& q, int cell,
                                             const DevBufs& b) {
    if (k.emit == 1) {
        store_moments<C>(q, cell, b);
    } else if (k.emit == 2) {
        b.rho[cell] += 1.0 + (double)q.drho;
        b.ux[cell] += (double)q.ux;
        b.uy[cell] += (double)q.uy;
    }
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
    if (ys < 0) return fill_val<S, C>(k, pb, A);
    if (ys >= k.Ny) return fill_val<S, C>(k, pt, A);
    int xs = x - k.sx[A];
    xs += (xs < 0) ? k.Nx : 0;
    return ld_val<S, C>(src[(long long)A * k.plane + (long long)ys * k.Nx + xs]);
}

template <class SET, typename S, typename C, int... I>
__device__ __forceinline__ void pull_wall_ct(const KParams<C>& k, const S* __restrict__ src, int x,
                                             int y, C* f, std::integer_sequence<int, I...>) {
    const C pb = y < k.maxey ? C(wall_dpsi_ct<SET, S, C, true>(k, src, x)) : C(0);
    const C pt = y >= k.Ny - k.maxey ? C(wall_dpsi_ct<SET, S, C, false>(k, src, x)) : C(0);
    ((f[I] = wall_value<SET, S, C, I>(k, src, x, y, pb, pt)), ...);
}

// e_y of plane a of a compiled set (rest, the P pair members, their negatives)
template <class SET>
__host__ __device__ constexpr int plane_ey_ct(int a) {
    return a < SET::R ? 0 : (a < SET::R + SET::P ? SET::ey[a - SET::R] : -SET::ey[a - SET::R - SET::P]);
}

// Populations of a node in the four rows next to one wall, the wall's dPsi
// given: the fill where the source lies beyond that wall, the pull otherwise
// (the other wall is out of reach, Ny >= 8).
template <class SET, typename S, typename C, bool BOTTOM, int A>
__device__ __forceinline__ C strip_value(const KParams<C>& k, const S* __restrict__ src, int x, int y,
                                         C dpsi) {
    constexpr int EY = plane_ey_ct<SET>(A);
    const int ys = y - EY;
    if (BOTTOM ? ys < 0 : ys >= k.Ny) return fill_val<S, C>(k, dpsi, A);
    int xs = x - k.sx[A];
    xs += (xs < 0) ? k.Nx : 0;
    return ld_val<S, C>(src[(long long)A * k.plane + (long long)ys * k.Nx + xs]);
}

template <class SET, typename S, typename C, bool BOTTOM, int... I>
__device__ __forceinline__ void strip_values(const KParams<C>& k, const S* __restrict__ src, int x, int y,
                                             C dpsi, C* f, std::integer_sequence<int, I...>) {
    ((f[I] = strip_value<SET, S, C, BOTTOM, I>(k, src, x, y, dpsi)), ...);
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

// The same sums from h = d / (w S) (16-bit storage): d = w S h, so every
// term is weighed with the pair's w S e... constants.
template <int EX, int EY, typename C>
__device__ __forceinline__ void moment_pair_h(const KParams<C>& k, int p, C fp, C fm, C& drho,
                                              C& Jx, C& Jy, C& Kxx, C& Kxy, C& Kyy) {
    const C sum = fp + fm, dif = fp - fm;
    drho = fma(k.hw[p], sum, drho);
    if constexpr (EX != 0) Jx = fma(k.hwx[p], dif, Jx);
    if constexpr (EY != 0) Jy = fma(k.hwy[p], dif, Jy);
    if constexpr (EX != 0) Kxx = fma(k.hwxx[p], sum, Kxx);
    if constexpr (EX * EY != 0) Kxy = fma(k.hwxy[p], sum, Kxy);
    if constexpr (EY != 0) Kyy = fma(k.hwyy[p], sum, Kyy);
}

// Deviation moments drho = sum d, J = sum d e, K = sum d e e of the node's
// register values (d, or h for 16-bit storage).
template <class SET, typename S, typename C, int... I>
__device__ __forceinline__ void moments_ct(const KParams<C>& k, const C* f, C& drho, C& Jx, C& Jy,
                                           C& Kxx, C& Kxy, C& Kyy, std::integer_sequence<int, I...>) {
    if constexpr (Storage<S>::scaled) {
        drho = SET::R ? mul_rn(k.hw_rest, f[0]) : C(0);
        (moment_pair_h<SET::ex[I], SET::ey[I], C>(k, I, f[SET::R + I], f[SET::R + SET::P + I], drho,
                                                  Jx, Jy, Kxx, Kxy, Kyy), ...);
    } else {
        drho = SET::R ? f[0] : C(0);
        (moment_pair<SET::ex[I], SET::ey[I], C>(f[SET::R + I], f[SET::R + SET::P + I], drho, Jx, Jy,
                                                Kxx, Kxy, Kyy), ...);
    }
}

// ---- relaxation of a compiled set: the target as polynomials in e -----------
// With s = (c u).e and t = s^2, the relaxation target of Eq. nm.3 / nm.4
// (feq/w - 1 = even + odd part, as in pair_update) is a polynomial in the
// integer components (ex, ey) of the positive pair member:
//   Ge = c00 + c20 ex^2 + c11 ex ey + c02 ey^2
//        + c40 ex^4 + c31 ex^3 ey + c22 ex^2 ey^2 + c13 ex ey^3 + c04 ey^4
//   Go = d10 ex + d01 ey + d30 ex^3 + d21 ex^2 ey + d12 ex ey^2 + d03 ey^3
// whose node coefficients follow from expanding a0 + a1 t + a2 t^2 and
// s (b0 + b1 t) in X = c u_x, Y = c u_y, plus the force terms (g along x):
// tau rho (g.xi) s adds trcg X to c20 and trcg Y to c11; the odd force part
// e_x (k0 + cqxx ex^2 + 2 cqxy ex ey + cqyy ey^2) - (hx ex + hy ey) adds
// k0 - hx to d10, cqxx to d30, 2 cqxy to d21, cqyy to d12 and -hy to d01.
// Per pair the integer powers of e are compile-time constants, so the force
// costs nothing per population, and the pairs that share (|ex|, |ey|) share
// their partial sums:  Ge = Ee + sx sy Eo,  Go = sx Ox + sy Oy  with
// sx, sy the signs of ex, ey and Ee, Eo, Ox, Oy the parts of Ge, Go even in
// both, odd in both, odd in ex only, odd in ey only.
template <typename C>
struct PolyCoef {
    C c00, c20, c11, c02, c40, c31, c22, c13, c04;
    C d10, d01, d30, d21, d12, d03;
};

// sc scales every coefficient (1: deviation units; omega / S: 16-bit units)
template <int N, bool FORCE, bool SCALE, typename C>
__device__ __forceinline__ PolyCoef<C> poly_coef(const CellCoef<C>& q, C sc) {
    const C X = q.utx, Y = q.uty;
    const C X2 = mul_rn(X, X), Y2 = mul_rn(Y, Y), XY = mul_rn(X, Y);
    PolyCoef<C> p{};
    p.c00 = q.a0;
    p.c20 = mul_rn(q.a1, X2);
    p.c11 = mul_rn(C(2) * q.a1, XY);
    p.c02 = mul_rn(q.a1, Y2);
    if constexpr (FORCE) {
        p.c20 = fma(q.trcg, X, p.c20);
        p.c11 = fma(q.trcg, Y, p.c11);
    }
    if constexpr (N >= 4) {
        const C a2 = q.a2;
        p.c40 = mul_rn(a2, mul_rn(X2, X2));
        p.c31 = mul_rn(C(4) * a2, mul_rn(X2, XY));
        p.c22 = mul_rn(C(6) * a2, mul_rn(X2, Y2));
        p.c13 = mul_rn(C(4) * a2, mul_rn(XY, Y2));
        p.c04 = mul_rn(a2, mul_rn(Y2, Y2));
    }
    p.d10 = mul_rn(q.b0, X);
    p.d01 = mul_rn(q.b0, Y);
    if constexpr (N >= 3) {
        const C b1 = q.b1;
        p.d30 = mul_rn(b1, mul_rn(X, X2));
        p.d21 = mul_rn(C(3) * b1, mul_rn(X2, Y));
        p.d12 = mul_rn(C(3) * b1, mul_rn(X, Y2));
        p.d03 = mul_rn(b1, mul_rn(Y, Y2));
    }
    if constexpr (FORCE) {
        p.d10 = p.d10 + (q.k0 - q.hx);
        p.d01 = p.d01 - q.hy;
        if constexpr (N >= 3) {
            p.d30 = p.d30 + q.cqxx;
            p.d21 = p.d21 + C(2) * q.cqxy;
            p.d12 = p.d12 + q.cqyy;
        }
    }
    if constexpr (SCALE) {
        C* v = &p.c00;
#pragma unroll
        for (int i = 0; i < 15; ++i) v[i] = mul_rn(v[i], sc);
    }
    return p;
}

template <int K, typename C>
__device__ __forceinline__ C muli(C v) {          // K v, K > 0
    if constexpr (K == 1) return v;
    else return mul_rn(C(K), v);
}

template <int K, typename C>
__device__ __forceinline__ C fmai(C a, C v) {     // a + K v, K >= 0
    if constexpr (K == 0) return a;
    else if constexpr (K == 1) return a + v;
    else return fma(C(K), v, a);
}

// Parts of Ge, Go for |ex| = AX, |ey| = AY (see PolyCoef).
template <int AX, int AY, int N, typename C>
struct PolyParts {
    C Ee, Eo, Ox, Oy;
    __device__ __forceinline__ explicit PolyParts(const PolyCoef<C>& p) {
        Ee = fmai<AX * AX>(p.c00, p.c20);
        Ee = fmai<AY * AY>(Ee, p.c02);
        if constexpr (N >= 4) {
            Ee = fmai<AX * AX * AX * AX>(Ee, p.c40);
            Ee = fmai<AX * AX * AY * AY>(Ee, p.c22);
            Ee = fmai<AY * AY * AY * AY>(Ee, p.c04);
        }
        Eo = C(0);
        if constexpr (AX * AY != 0) {
            Eo = muli<AX * AY>(p.c11);
            if constexpr (N >= 4) {
                Eo = fmai<AX * AX * AX * AY>(Eo, p.c31);
                Eo = fmai<AX * AY * AY * AY>(Eo, p.c13);
            }
        }
        Ox = C(0);
        if constexpr (AX != 0) {
            Ox = muli<AX>(p.d10);
            if constexpr (N >= 3) {
                Ox = fmai<AX * AX * AX>(Ox, p.d30);
                Ox = fmai<AX * AY * AY>(Ox, p.d12);
            }
        }
        Oy = C(0);
        if constexpr (AY != 0) {
            Oy = muli<AY>(p.d01);
            if constexpr (N >= 3) {
                Oy = fmai<AX * AX * AY>(Oy, p.d21);
                Oy = fmai<AY * AY * AY>(Oy, p.d03);
            }
        }
    }
};

__host__ __device__ constexpr int iabs(int v) { return v < 0 ? -v : v; }

// First pair of a compiled set with the same (|ex|, |ey|) as pair p.
template <class SET>
__host__ __device__ constexpr int poly_class(int p) {
    for (int q = 0; q < p; ++q)
        if (iabs(SET::ex[q]) == iabs(SET::ex[p]) && iabs(SET::ey[q]) == iabs(SET::ey[p])) return q;
    return p;
}

// Relax pair J (a member of the class of pair P0) from the class's parts.
// Deviation units: d* = (1 - omega) d + omega w (Ge +- Go); 16-bit units
// (coefficients already times omega / S): h* = (1 - omega) h + (Ge +- Go).
template <class SET, int J, bool HSPACE, typename C, class PARTS>
__device__ __forceinline__ void poly_pair(const KParams<C>& k, const PARTS& pp, C* f) {
    constexpr int EX = SET::ex[J], EY = SET::ey[J];
    constexpr bool nx = EX < 0, ny = EY < 0;
    const C Ge = (nx != ny) ? pp.Ee - pp.Eo : pp.Ee + pp.Eo;
    C Go;
    if constexpr (EX == 0) Go = ny ? -pp.Oy : pp.Oy;
    else if constexpr (EY == 0) Go = nx ? -pp.Ox : pp.Ox;
    else Go = nx ? (ny ? -(pp.Ox + pp.Oy) : pp.Oy - pp.Ox) : (ny ? pp.Ox - pp.Oy : pp.Ox + pp.Oy);
    C& fp = f[SET::R + J];
    C& fm = f[SET::R + SET::P + J];
    const C omo = k.one_m_omega;
    if constexpr (HSPACE) {
        fp = fma(omo, fp, Ge + Go);
        fm = fma(omo, fm, Ge - Go);
    } else {
        const C omw = k.pomw[J];
        const C Xe = mul_rn(omw, Ge);
        fp = fma(omo, fp, fma(omw, Go, Xe));
        fm = fma(omo, fm, fma(-omw, Go, Xe));
    }
}

template <class SET, int P0, int N, bool HSPACE, typename C, int... J>
__device__ __forceinline__ void poly_class_relax(const KParams<C>& k, const PolyCoef<C>& pc, C* f,
                                                 std::integer_sequence<int, J...>) {
    if constexpr (poly_class<SET>(P0) == P0) {
        const PolyParts<iabs(SET::ex[P0]), iabs(SET::ey[P0]), N, C> pp(pc);
        ((poly_class<SET>(J) == P0 ? poly_pair<SET, J, HSPACE, C>(k, pp, f) : void()), ...);
    }
}

template <class SET, int N, bool HSPACE, typename C, int... I>
__device__ __forceinline__ void poly_relax_all(const KParams<C>& k, const PolyCoef<C>& pc, C* f,
                                               std::integer_sequence<int, I...> seq) {
    (poly_class_relax<SET, I, N, HSPACE, C>(k, pc, f, seq), ...);
}

// Force-free relaxation of the pair (+e, -e), e = (EX, EY) known at compile
// time, in the per-pair form: s = (c u).e, t = s^2, Ge = a0 + t (a1 + t a2),
// Go = s (b0 + t b1).  Without the force terms this costs fewer operations
// per pair than the polynomial form's shared partial sums.
template <int EX, int EY, int N, bool HSPACE, typename C>
__device__ __forceinline__ void pair_update_free(const CellCoef<C>& q, C omw, C omo, C sc, C& fp,
                                                 C& fm) {
    const C s = lin<EX, EY>(q.utx, q.uty);
    const C t = mul_rn(s, s);
    const C Ge = N >= 4 ? fma(t, fma(t, q.a2, q.a1), q.a0) : fma(t, q.a1, q.a0);
    const C Go = N >= 3 ? mul_rn(s, fma(t, q.b1, q.b0)) : mul_rn(s, q.b0);
    if constexpr (HSPACE) {          // sc = omega / S
        const C Xe = mul_rn(sc, Ge);
        fp = fma(omo, fp, fma(sc, Go, Xe));
        fm = fma(omo, fm, fma(-sc, Go, Xe));
    } else {
        const C Xe = mul_rn(omw, Ge);
        fp = fma(omo, fp, fma(omw, Go, Xe));
        fm = fma(omo, fm, fma(-omw, Go, Xe));
    }
}

template <class SET, int N, bool HSPACE, typename C, int... I>
__device__ __forceinline__ void relax_free_all(const KParams<C>& k, const CellCoef<C>& q, C* f,
                                               std::integer_sequence<int, I...>) {
    const C sc = HSPACE ? k.om_s : C(1);
    (pair_update_free<SET::ex[I], SET::ey[I], N, HSPACE, C>(q, k.pomw[I], k.one_m_omega, sc,
                                                            f[SET::R + I], f[SET::R + SET::P + I]),
     ...);
}

// Relaxation of every population of a node of a compiled set (Eq. nm.8 with
// feq = f0 + tau F, Eq. nm.2-nm.4), in place on the register values: the
// polynomial form with the force, the per-pair form without it.
template <class SET, int N, typename S, typename C>
__device__ __forceinline__ void relax_ct(const KParams<C>& k, const CellCoef<C>& q, C* f) {
    constexpr bool H = Storage<S>::scaled;
    if (k.force) {
        const PolyCoef<C> pc = poly_coef<N, true, H, C>(q, H ? k.om_s : C(1));
        if constexpr (SET::R) {
            if constexpr (H) f[0] = fma(k.one_m_omega, f[0], pc.c00);
            else f[0] = fma(k.one_m_omega, f[0], k.omw_rest * q.a0);
        }
        poly_relax_all<SET, N, H, C>(k, pc, f, std::make_integer_sequence<int, SET::P>{});
    } else {
        if constexpr (SET::R) {
            if constexpr (H) f[0] = fma(k.one_m_omega, f[0], mul_rn(k.om_s, q.a0));
            else f[0] = fma(k.one_m_omega, f[0], k.omw_rest * q.a0);
        }
        relax_free_all<SET, N, H, C>(k, q, f, std::make_integer_sequence<int, SET::P>{});
    }
}

// Stored values of a node's post-collision register values.  16-bit storage
// rounds stochastically, two values per conversion: the rest value with a
// zero partner, then each +-e pair, with the random bits r0 + (p + 1) phi
// (r0 the node's hash, phi = 0x9e3779b9) -- a function of (node, step,
// pair) only, so every kernel that packs a node this way stores its bits.
template <class SET, typename S, typename C>
__device__ __forceinline__ void pack_ct(const C* f, unsigned r0, S* out) {
    constexpr int R = SET::R, P = SET::P, V = R + 2 * P;
    if constexpr (Storage<S>::scaled) {
        if constexpr (R) {
            S zero;
            Storage<S>::sr2(f[0], 0.f, r0, out[0], zero);
        }
#pragma unroll
        for (int p = 0; p < P; ++p)
            Storage<S>::sr2(f[R + p], f[R + P + p], r0 + unsigned(p + 1) * 0x9e3779b9u, out[R + p],
                            out[R + P + p]);
    } else {
#pragma unroll
        for (int a = 0; a < V; ++a) out[a] = S(f[a]);
    }
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
        f[a] = ld_val<S, C>(static_cast<const S*>(sp[a])[i]);
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
    return ld_val<S, C>(ld_stream(static_cast<const S*>(sp[A]) + i));
}

template <class SET, typename S, typename C, int A, class PTR>
__device__ __forceinline__ C pull_col1(const KParams<C>& k, const PTR& sp, int cell) {
    return ld_val<S, C>(ld_stream(static_cast<const S*>(sp[A]) + cell + plane_ex<SET>(A)));
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

// ---- wall strips ------------------------------------------------------------
// With four wall rows (max|e_y| = 4) every node of the rows 0..3 of a column
// needs the same flux balance dPsi(x) of its wall, which wall_dpsi_ct sums
// from ~26 fp64 terms on four interleaved accumulators (term t into
// accumulator t mod 4).  A strip block covers 32 columns x the 4 wall rows of
// one wall: warp r (one row) sums accumulator r's terms for its 32 columns,
// in the same order, and the four partial sums meet in shared memory as
// (a0 + a1) + (a2 + a3): the bits of wall_dpsi_ct at a quarter of the work.

template <class SET, bool BOTTOM, int RR, class TERM, int A>
__device__ __forceinline__ void strip_add_plane(double& acc, const TERM& term) {
    constexpr int ey = plane_ey_ct<SET>(A);
    if constexpr (BOTTOM ? ey < 0 : ey > 0) {
        constexpr int n = BOTTOM ? -ey : ey;
        constexpr int t0 = wall_terms_before<SET, BOTTOM>(A);
#pragma unroll
        for (int j = 0; j < n; ++j)
            if (((t0 + j) & 3) == RR) acc += term(std::integral_constant<int, A>{}, j);
    }
}

template <class SET, bool BOTTOM, int RR, class TERM, int... I>
__device__ __forceinline__ double strip_partial(const TERM& term, std::integer_sequence<int, I...>) {
    double acc = 0.0;
    (strip_add_plane<SET, BOTTOM, RR, TERM, I>(acc, term), ...);
    return acc;
}

template <class SET, int N, typename S, typename C, bool BOTTOM>
__device__ __forceinline__ void wall_strip(const KParams<C>& k, const S* __restrict__ src, int strip,
                                           const DevBufs& b) {
    constexpr int R = SET::R, P = SET::P, V = R + 2 * P;
    __shared__ double part[4][32];
    const int r = threadIdx.x >> 5;                 // warp = wall row offset (nearest first)
    const int lane = threadIdx.x & 31;
    const int x = strip * 32 + lane;
    const int y = BOTTOM ? r : k.Ny - 1 - r;
    auto term = [&](auto bc, int j) {
        constexpr int bb = decltype(bc)::value;
        int xs = x - k.sx[bb];
        xs += (xs < 0) ? k.Nx : 0;
        const int row = BOTTOM ? j : (k.Ny - 1 - j);
        return (double)ld_pop<S, C>(k, src[(long long)bb * k.plane + (long long)row * k.Nx + xs], bb);
    };
    constexpr auto seq = std::make_integer_sequence<int, V>{};
    double acc;
    switch (r) {                                    // warp-uniform
        case 0: acc = strip_partial<SET, BOTTOM, 0>(term, seq); break;
        case 1: acc = strip_partial<SET, BOTTOM, 1>(term, seq); break;
        case 2: acc = strip_partial<SET, BOTTOM, 2>(term, seq); break;
        default: acc = strip_partial<SET, BOTTOM, 3>(term, seq); break;
    }
    part[r][lane] = acc;
    __syncthreads();
    const C dpsi = C(((part[0][lane] + part[1][lane]) + (part[2][lane] + part[3][lane])) * k.inv_den);
    const int cell = y * k.Nx + x;
    C f[V];
    strip_values<SET, S, C, BOTTOM>(k, src, x, y, dpsi, f, seq);
    C drho, Jx = 0, Jy = 0, Kxx = 0, Kxy = 0, Kyy = 0;
    moments_ct<SET, S, C>(k, f, drho, Jx, Jy, Kxx, Kxy, Kyy, std::make_integer_sequence<int, P>{});
    const CellCoef<C> q = cell_coef<N, C>(k, drho, Jx, Jy, Kxx, Kxy, Kyy);
    relax_ct<SET, N, S, C>(k, q, f);
    S out[V];
    pack_ct<SET, S, C>(f, sr_seed<S, C>(k.seed, cell), out);
#pragma unroll
    for (int a = 0; a < V; ++a) static_cast<S*>(k.dstp[a])[cell] = out[a];
    emit_moments<C>(k, q, cell, b);
    flag_density<C>(q, b.status);
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
    // With wall strips the grid starts with the bottom and the top strips (the
    // heavier blocks run first, the uniform interior blocks form the tail);
    // block 2 strips + m then takes the interior block at node (strips + m) 128.
    int blk = int(blockIdx.x);
    if (k.strips) {
        if (blk < k.strips) {
            wall_strip<SET, N, S, C, true>(k, src, blk, b);
            return;
        }
        if (blk < 2 * k.strips) {
            wall_strip<SET, N, S, C, false>(k, src, blk - k.strips, b);
            return;
        }
        blk -= k.strips;
    }
    const int c0 = blk * kBlock;
    const int cell = c0 + threadIdx.x;
    const int y0 = c0 / k.Nx;
    const int x0 = c0 - y0 * k.Nx;
    const bool fast = x0 >= k.maxex && x0 + kBlock - 1 + k.maxex < k.Nx && y0 >= k.maxey &&
                      y0 < k.Ny - k.maxey;
    const int y1 = (min(c0 + kBlock, k.ncell) - 1) / k.Nx;
    const bool rows = !fast && y0 >= k.maxey && y1 < k.Ny - k.maxey;
    bool wfast = fast;
    if (rows) {   // a warp of one row away from both x ends pulls at fixed offsets
        const int y = cell / k.Nx, x = cell - y * k.Nx;
        const int ylead = __shfl_sync(0xffffffffu, y, 0);
        wfast = __all_sync(0xffffffffu, cell < k.ncell && x >= k.maxex && x < k.Nx - k.maxex &&
                                            y == ylead);
    }
    C f[V];
    if (wfast) {
#pragma unroll
        for (int a = 0; a < V; ++a) f[a] = ld_val<S, C>(ld_stream(static_cast<const S*>(k.srcf[a]) + cell));
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
    C drho, Jx = 0, Jy = 0, Kxx = 0, Kxy = 0, Kyy = 0;
    moments_ct<SET, S, C>(k, f, drho, Jx, Jy, Kxx, Kxy, Kyy, std::make_integer_sequence<int, P>{});
    const CellCoef<C> q = cell_coef<N, C>(k, drho, Jx, Jy, Kxx, Kxy, Kyy);
    relax_ct<SET, N, S, C>(k, q, f);
    S out[V];
    pack_ct<SET, S, C>(f, sr_seed<S, C>(k.seed, cell), out);
#pragma unroll
    for (int a = 0; a < V; ++a) static_cast<S*>(k.dstp[a])[cell] = out[a];
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
