// TM walk: a diffusion coefficient that jumps across vertical interfaces.
//
// Sub-domains are vertical strips; strip m = [xif[m-1], xif[m]) has diffusion
// D_m and rates kappa_{e,m}, so D_m Lap u = i kappa_{e,m} u there, with the
// flux D du/dn continuous across interfaces (Sec. 2.2, the Helmholtz
// equation per sub-domain).  One step from beta in strip i (Sec. 3.1):
//   1. beta' = beta + sqrt(D_i dt) W (the discretised-process equation);
//   2. the outer boundary first: overshoot, or the Brownian-bridge test with
//      kappa_i = D_i, 2 d d' / (D_i dt) <= -ln U;
//   3. interfaces to a strip of other D (equal D: no regime change): crossed
//      -> hitting fraction |d / (beta'_x - beta_x)|; not crossed -> the
//      bridge test against the nearer interface with its own uniform U_g.
//      A hit at fraction th resumes on side i with probability
//      p_i = D_i / (D_i + D_j) (the crossing-probability equation), uniformly
//      in the disc of radius h = sqrt(dt max(D_i, D_j)) tangent to the
//      interface at the hit height on that side, and splits the step's time:
//      side i: T_i += 1 - (1 - th) p_i / 2, T_j += (1 - th) p_i / 2;
//      side j: T_i += th + (1 - th) p_j / 2, T_j the rest of the step.  A
//      resampled point outside the domain ends the walk on the nearest wall.
//   4. otherwise the step's time goes to the strip of beta'.
// A walk that starts on an interface has hit it at time 0 (from the left).
// Random numbers: the step's normals and wall-bridge uniform as in the TE
// walk of the same precision; U_g, U_alpha and the disc's radius and angle
// from the Philox call with counter (n, path, node, 2).
//
// Real = double is the parity walk (absolute coordinates, the order of
// operations of the definition, compiled without contraction); Real = float
// is the throughput walk on the single-precision stream.  Occupation times
// (units of dt) are kept per lane in shared memory.
#pragma once

#include "walk_sched.cuh"

namespace sdd {

template <class Real_, int KMAX_>
struct WalkerTM {
    using Real = Real_;
    static constexpr int KMAX = KMAX_;
    static constexpr bool kF64 = sizeof(Real) == 8;
    static constexpr bool kCoop = false;
    using Occ = Real;  // occupation time of every strip
    using HistT = Real;
    static constexpr int kStored = KMAX;
    static constexpr int kHist = KMAX;

    Real x, z;
    int i;             // strip of (x, z)
    uint32_t n;        // steps taken
    uint32_t hits;     // interface randomisations
    uint32_t nid, path_;
    uint32_t pre_x, pre_y;
    bool start_on_if;
    Real *h;           // this lane's occupation times: h[32 m] for strip m

    __device__ __forceinline__ void bind(HistT *p) { h = p; }

    __device__ __forceinline__ static Real xif(const ModelDev &M, int k) {
        if constexpr (kF64) return M.xif[k]; else return M.fxif[k];
    }
    __device__ __forceinline__ static Real diff(const ModelDev &M, int k) {
        if constexpr (kF64) return M.diff[k]; else return M.fdiff[k];
    }
    __device__ __forceinline__ static int strip(const ModelDev &M, Real xx) {
        int k = 0;
        while (k < M.K - 1 && xx >= xif(M, k)) ++k;
        return k;
    }

    __device__ __forceinline__ void start(const ModelDev &M, const WalkArgs &A, double x0, double z0,
                                          uint32_t path, uint32_t node_id, int) {
        x = (Real)x0;
        z = (Real)z0;
        i = strip(M, x);
        n = 0;
        hits = 0;
        nid = node_id;
        path_ = path;
        pre_x = __umulhi(0xCD9E8D57u, node_id) ^ path ^ A.rk0[0];
        pre_y = 0xCD9E8D57u * node_id;
        start_on_if = i > 0 && x == xif(M, i - 1) && diff(M, i - 1) != diff(M, i);
#pragma unroll
        for (int k = 0; k < KMAX; ++k) h[32 * k] = Real(0);
    }

    __device__ __forceinline__ void counts(Occ *c) const {
#pragma unroll
        for (int k = 0; k < KMAX; ++k) c[k] = h[32 * k];
    }

    // uniforms of the precision's stream
    __device__ __forceinline__ static Real uni(uint32_t w) {
        if constexpr (kF64) return ((double)w + 0.5) * (1.0 / 4294967296.0);
        else return ((float)(w & 0x7fffffu) + 0.5f) * (1.0f / 8388608.0f);
    }
    __device__ __forceinline__ Real wall_uniform(const WalkArgs &A, uint32_t wa, uint32_t wb) const {
        if constexpr (kF64) {
            const uint4 v = philox4x32_10(make_uint4(n, path_, nid, 1u), A.key0, A.key1);
            return uni(v.x);
        } else {
            return ((float)(((wa >> 23) << 9) | (wb >> 23)) + 0.5f) * (1.0f / 262144.0f);
        }
    }

    __device__ __forceinline__ void exit_at(ExitInfo<Real> &ei, Real ex, Real ez, Real th, int wall) {
        ei.x = ex;
        ei.z = ez;
        ei.th = th;
        ei.wall = wall;
        ei.mlast = i;
        ei.nocc = n;
        ei.aux = hits;
    }

    // One step driven by the Philox words (wa, wb) of step n.  Returns true
    // when the walk ended.
    __device__ __forceinline__ bool step(const ModelDev &M, const WalkArgs &A, uint32_t wa, uint32_t wb,
                                         ExitInfo<Real> &ei) {
        const Real dt = (Real)A.dt;
        Real Di = diff(M, i);
        Real xn, zn, th = Real(2), xg = Real(0);
        int side = -1, j = i;
        if (n == 0 && start_on_if) {
            i = i - 1;
            Di = diff(M, i);
            xn = x;
            zn = z;
            th = Real(0);
            side = i + 1;
            xg = x;
        } else {
            Real w0, w1;
            if constexpr (kF64) {
                const double rho = sqrt(-2.0 * log(uni(wa)));
                const double ang = 6.283185307179586 * uni(wb);
                w0 = rho * cos(ang);
                w1 = rho * sin(ang);
            } else {
                float sn, cs;
                const float rho = sqrtf(-2.0f * __logf(uni(wa)));
                __sincosf(6.28318530718f * uni(wb), &sn, &cs);
                w0 = rho * cs;
                w1 = rho * sn;
            }
            const Real s = sqrt(Di * dt);
            xn = x + s * w0;
            zn = z + s * w1;
            // 2. the outer boundary, with the strip's diffusion
            const Real d[4] = {x - (Real)M.xmin, (Real)M.xmax - x, z - (Real)M.zmin, (Real)M.zmax - z};
            const Real e[4] = {xn - (Real)M.xmin, (Real)M.xmax - xn, zn - (Real)M.zmin, (Real)M.zmax - zn};
            const bool over = e[0] <= Real(0) || e[1] <= Real(0) || e[2] <= Real(0) || e[3] <= Real(0);
            if (over) {
                Real best = Real(3);
                int bw = -1;
#pragma unroll
                for (int w = 0; w < 4; ++w)
                    if (e[w] <= Real(0)) {
                        const Real t = d[w] / (d[w] - e[w]);
                        if (bw < 0 || t < best) { best = t; bw = w; }
                    }
                place(M, xn, zn, best, bw, ei);
                return true;
            }
            const Real dtD = Di * dt;
            Real best = Real(0);
            int bw = -1;
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const Real q = Real(2) * d[w] * e[w] / dtD;
                if (bw < 0 || q < best) { best = q; bw = w; }
            }
            if (best <= Real(40)) {  // -ln U <= 33 ln 2 for every uniform of either stream
                const Real U = wall_uniform(A, wa, wb);
                const Real L = -log(U);
                if (best <= L) {
                    place(M, xn, zn, best / L, bw, ei);
                    return true;
                }
            }
            // 3. the interfaces of strip i
            j = strip(M, xn);
            if (j != i) {
                const int jn = j > i ? i + 1 : i - 1;
                const Real xi = j > i ? xif(M, i) : xif(M, i - 1);
                if (diff(M, jn) != Di) {
                    th = fabs((x - xi) / (xn - x));
                    side = jn;
                    xg = xi;
                }
            } else {
                Real bq = Real(0), bx = Real(0);
                int bs = -1;
                if (i > 0 && diff(M, i - 1) != Di) {
                    const Real xl = xif(M, i - 1);
                    bq = Real(2) * (x - xl) * (xn - xl) / dtD;
                    bs = i - 1;
                    bx = xl;
                }
                if (i < M.K - 1 && diff(M, i + 1) != Di) {
                    const Real xr = xif(M, i);
                    const Real q = Real(2) * (xr - x) * (xr - xn) / dtD;
                    if (bs < 0 || q < bq) { bq = q; bs = i + 1; bx = xr; }
                }
                if (bs >= 0 && bq <= Real(40)) {
                    const uint4 v = philox4x32_10(make_uint4(n, path_, nid, 2u), A.key0, A.key1);
                    const Real L = -log(uni(v.x));
                    if (bq <= L) {
                        th = bq / L;
                        side = bs;
                        xg = bx;
                    }
                }
            }
        }
        if (side >= 0) {
            const uint4 v = philox4x32_10(make_uint4(n, path_, nid, 2u), A.key0, A.key1);
            const Real Dj = diff(M, side);
            const Real pi_ = Di / (Di + Dj), pj = Dj / (Di + Dj);
            const Real zg = z + th * (zn - z);
            const Real hh = sqrt(dt * (Di > Dj ? Di : Dj));
            const Real c = x <= xg ? hh : -hh;
            const Real rest = Real(1) - th;
            Real cx;
            if (uni(v.y) < pi_) {
                h[32 * i] += Real(1) - Real(0.5) * rest * pi_;
                h[32 * side] += Real(0.5) * rest * pi_;
                cx = xg - c;
            } else {
                const Real ti = th + Real(0.5) * rest * pj;
                h[32 * i] += ti;
                h[32 * side] += Real(1) - ti;
                cx = xg + c;
            }
            const Real rho = hh * sqrt(uni(v.z));
            Real sa, ca;
            if constexpr (kF64) {
                const double ang = 6.283185307179586 * uni(v.w);
                ca = cos(ang);
                sa = sin(ang);
            } else {
                __sincosf(6.28318530718f * uni(v.w), &sa, &ca);
            }
            xn = cx + rho * ca;
            zn = zg + rho * sa;
            hits += 1;
            const Real e[4] = {xn - (Real)M.xmin, (Real)M.xmax - xn, zn - (Real)M.zmin, (Real)M.zmax - zn};
            int bw = -1;
            Real most = Real(0);
#pragma unroll
            for (int w = 0; w < 4; ++w)
                if (e[w] <= most && (bw < 0 || e[w] < most)) { most = e[w]; bw = w; }
            if (bw >= 0) {
                Real ex = xn < (Real)M.xmin ? (Real)M.xmin : (xn > (Real)M.xmax ? (Real)M.xmax : xn);
                Real ez = zn < (Real)M.zmin ? (Real)M.zmin : (zn > (Real)M.zmax ? (Real)M.zmax : zn);
                if (bw == 0) ex = (Real)M.xmin;
                if (bw == 1) ex = (Real)M.xmax;
                if (bw == 2) ez = (Real)M.zmin;
                if (bw == 3) ez = (Real)M.zmax;
                exit_at(ei, ex, ez, Real(0), bw);
                return true;
            }
            x = xn;
            z = zn;
            i = strip(M, x);
            n += 1;
            return false;
        }
        // 4. the step's time goes to the strip of beta'
        h[32 * j] += Real(1);
        x = xn;
        z = zn;
        i = j;
        n += 1;
        return false;
    }

    __device__ __forceinline__ void place(const ModelDev &M, Real xn, Real zn, Real th, int w,
                                          ExitInfo<Real> &ei) {
        Real ex = x + th * (xn - x), ez = z + th * (zn - z);
        if (w == 0) ex = (Real)M.xmin;
        if (w == 1) ex = (Real)M.xmax;
        if (w == 2) ez = (Real)M.zmin;
        if (w == 3) ez = (Real)M.zmax;
        exit_at(ei, ex, ez, th, w);
    }

    // The steps of one Philox call (two, or one when n is odd after a walk
    // started on an interface).  0 running, 1 exited, 2 truncated.
    __device__ __forceinline__ int iterate(const ModelDev &M, const WalkArgs &A, uint32_t,
                                           ExitInfo<Real> &ei) {
        const uint4 w = philox_rk_pre(n >> 1, 0u, pre_x, pre_y, A.rk0, A.rk1);
        if ((n & 1u) == 0u && step(M, A, w.x, w.y, ei)) return 1;
        if (step(M, A, w.z, w.w, ei)) return 1;
        if (n >= A.max_steps) {
            exit_at(ei, x, z, Real(0), 0);
            return 2;
        }
        return 0;
    }

    __device__ static void to_abs(const ModelDev &, Real X, Real Z, double &ox, double &oz) {
        ox = (double)X;
        oz = (double)Z;
    }

    // Sample for evaluation e: g(exit) exp(-i (1/2) sum_m kappa_{e,m} T_m dt),
    // T_m the occupation times c[m] plus th for the strip of the last point.
    __device__ static double2 sample(const ModelDev &M, const SharedTables &T, const WalkArgs &A,
                                     int, int e, Real xe, Real ze, Real th, int wall, int mlast,
                                     const Occ *c) {
        const double dt = A.dt;
        const double *kap = T.kappa + e * M.K;
        double ph = 0.0;
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
            if (k < M.K) ph += kap[k] * ((double)c[k] * dt);
        ph += kap[mlast] * ((double)th * dt);
        ph *= 0.5;
        double sw, cw;
        if constexpr (kF64) {
            sincos(ph, &sw, &cw);
        } else {
            const double q = rint(ph * 0.15915494309189535);
            float s, co;
            sincosf((float)(ph - q * 6.283185307179586), &s, &co);
            sw = s;
            cw = co;
        }
        const double x = (double)xe, z = (double)ze;
        double gr, gi;
        if (M.g_kind == 1) {
            const double *a = M.g_coef;
            gr = a[0] + a[2] * x + a[4] * z;
            gi = a[1] + a[3] * x + a[5] * z;
        } else if (M.g_kind == 2) {
            gr = x * x - z * z;
            gi = 0.0;
        } else if (M.g_kind == 3) {
            // (z + 1) cosh(a x), a = sqrt(i kappa_{e,s} / D_s) for the strip s of x
            int s = 0;
            while (s < M.K - 1 && x >= M.xif[s]) ++s;
            const double p = M.tm_a[e][s][0] * x, q = M.tm_a[e][s][1] * x;
            gr = (z + 1.0) * (cosh(p) * cos(q));
            gi = (z + 1.0) * (sinh(p) * sin(q));
        } else {
            // int_{xmin}^x ds / D(s)
            double u = 0.0, a = M.xmin;
            gr = 0.0;
            for (int k = 0; k < M.K; ++k) {
                const double b = k < M.K - 1 ? M.xif[k] : M.xmax;
                if (x <= b) {
                    gr = u + (x - a) / M.diff[k];
                    break;
                }
                u += (b - a) / M.diff[k];
                a = b;
                gr = u;
            }
            gi = 0.0;
        }
        (void)wall;
        // (cw - i sw)(gr + i gi)
        return make_double2(cw * gr + sw * gi, cw * gi - sw * gr);
    }
};

}  // namespace sdd
