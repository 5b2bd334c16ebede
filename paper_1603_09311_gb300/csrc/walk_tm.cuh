// TM walk: a diffusion coefficient that jumps across vertical interfaces.
//
// Sub-domains are vertical strips; strip m = [xif[m-1], xif[m]) has diffusion
// D_m and rates kappa_{e,m}, so D_m Lap u = i kappa_{e,m} u there, with the
// flux D du/dn continuous across interfaces (Sec. 2.2, the Helmholtz
// equation per sub-domain).  One step from beta in strip i (Sec. 3.1):
//   1. beta' = beta + sqrt(D_i dt) W (the discretised-process equation);
//   2. the outer boundary first: overshoot, or the Brownian-bridge test with
//      kappa_i = D_i for the wall of smallest w = 2 d d' / (D_i dt): hit iff
//      U <= p_w = exp(-w), U the step's bridge uniform;
//   3. interfaces to a strip of other D (equal D: no regime change): crossed
//      -> hitting fraction |d / (beta'_x - beta_x)|; not crossed -> the
//      bridge test for the nearer interface, g = 2 d d' / (D_i dt), with the
//      uniform U_g = (U - p_w) / (1 - p_w) the wall test leaves: hit iff
//      U <= p_w + (1 - p_w) exp(-g), at fraction g / (-ln U_g).
//      A hit at fraction th resumes on side i with probability
//      p_i = D_i / (D_i + D_j) (the crossing-probability equation), uniformly
//      in the disc of radius h = sqrt(dt max(D_i, D_j)) tangent to the
//      interface at the hit height on that side, and splits the step's time:
//      side i: T_i += 1 - (1 - th) p_i / 2, T_j += (1 - th) p_i / 2;
//      side j: T_i += th + (1 - th) p_j / 2, T_j the rest of the step.  A
//      resampled point outside the domain ends the walk on the nearest wall.
//   4. otherwise the step's time goes to the strip of beta'.
// A walk that starts on an interface has hit it at time 0 (from the left).
// Random numbers: the step's normals and bridge uniform as in the TE walk of
// the same precision; U_alpha and the disc's radius and angle from words
// 1, 2, 3 of the Philox call with counter (n, path, node, 2).
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
    static constexpr bool kGrouped = false;
    static constexpr int kMinCTAs = 3;
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

    __device__ __forceinline__ void counts(const ModelDev &, uint32_t, Occ *c) const {
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
            const Real U = wall_uniform(A, wa, wb);
            const Real pw = best <= Real(40) ? exp(-best) : Real(0);
            if (U <= pw) {
                place(M, xn, zn, best / -log(U), bw, ei);
                return true;
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
                const Real pg = (bs >= 0 && bq <= Real(40)) ? exp(-bq) : Real(0);
                if (pg > Real(0) && U <= pw + (Real(1) - pw) * pg) {
                    th = bq / -log((U - pw) / (Real(1) - pw));
                    side = bs;
                    xg = bx;
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

// Throughput form of the single-precision TM walk: the same steps on the
// same stream as WalkerTM<float>, arranged like the TE walk.  Coordinates are
// centred (X = x - xc); the strip's step scale sqrt(D_i dt), filter
// thresholds and bounds live in registers and change only with the strip.
// A step takes the short path unless its wall product d d' or its product
// of distances to the strip's bounds comes within reach of a hit (or the
// step crossed a bound); the long path decides exactly as WalkerTM does.  A
// lane whose step needs the long path records that step; the steps it still
// runs in the iteration are discarded.  The long path and the interface
// randomisation then run once for all such lanes of the warp.  Whole steps in
// the current strip are counted in a register and added to the lane's
// occupation times when the strip changes or the walk ends.
template <int KMAX_>
struct WalkerTM32 {
    using Real = float;
    static constexpr int KMAX = KMAX_;
    static constexpr bool kCoop = false;
    static constexpr bool kGrouped = false;
    static constexpr int kMinCTAs = 3;
    using Occ = float;
    using HistT = float;
    static constexpr int kStored = KMAX;
    static constexpr int kHist = KMAX;
    // four Philox calls (8 steps) per round of an iteration: the per-step
    // code is the short path only (the long path and the events run once per
    // iteration), so the loop fits the instruction cache (measured with one
    // round: 1, 2, 4 calls -> 1.26e11, 1.50e11, 1.64e11 walk-steps/s on the
    // analytic test model)
    static constexpr int PAIRS = 4;

    float X, Z, dmin, dI;
    int i;
    uint32_t n, hits, run;
    uint32_t nid, path_, pre_x, pre_y;
    float s, wthr, c2, xl, xr, Di;
    float lc;  // -2 ln(2) D_i dt: squared step length = lc log2(u0)
    bool start_on_if;
    float *h;

    __device__ __forceinline__ void bind(HistT *p) { h = p; }

    __device__ __forceinline__ static int strip(const ModelDev &M, float Xc) {
        int k = 0;
        while (k < M.K - 1 && Xc >= M.fxif[k] - M.fxc) ++k;
        return k;
    }
    // the constants of strip i (bounds in centred coordinates)
    __device__ __forceinline__ void enter(const ModelDev &M, const WalkArgs &A, int k) {
        i = k;
        Di = M.fdiff[k];
        const float dtD = Di * (float)A.dt;
        s = sqrtf(dtD);
        lc = -1.38629436112f * dtD;
        // bands: out of both, p_w and p_g are below 2^-20 each, so no uniform
        // (>= 2^-19) can hit either: 2 d d' / (D dt) > 20 ln 2 (with a margin)
        wthr = 6.94f * 1.001f * dtD;
        c2 = 2.f / dtD;
        xl = k > 0 ? M.fxif[k - 1] - M.fxc : -3.0e38f;
        xr = k < M.K - 1 ? M.fxif[k] - M.fxc : 3.0e38f;
        dI = fminf(X - xl, xr - X);
    }
    __device__ __forceinline__ void flush() {
        h[32 * i] += (float)run;
        run = 0;
    }

    __device__ __forceinline__ void start(const ModelDev &M, const WalkArgs &A, double x0, double z0,
                                          uint32_t path, uint32_t node_id, int) {
        X = (float)x0 - M.fxc;
        Z = (float)z0 - M.fzc;
        dmin = fminf(M.fhw - fabsf(X), M.fhh - fabsf(Z));
        const float xa = (float)x0;
        int k = 0;
        while (k < M.K - 1 && xa >= M.fxif[k]) ++k;
        start_on_if = k > 0 && xa == M.fxif[k - 1] && M.fdiff[k - 1] != M.fdiff[k];
        enter(M, A, k);
        n = 0;
        hits = 0;
        run = 0;
        nid = node_id;
        path_ = path;
        pre_x = __umulhi(0xCD9E8D57u, node_id) ^ path ^ A.rk0[0];
        pre_y = 0xCD9E8D57u * node_id;
#pragma unroll
        for (int k2 = 0; k2 < KMAX; ++k2) h[32 * k2] = 0.f;
    }

    __device__ __forceinline__ void counts(const ModelDev &, uint32_t, Occ *c) const {
#pragma unroll
        for (int k = 0; k < KMAX; ++k) c[k] = h[32 * k];
    }

    __device__ __forceinline__ static float uni(uint32_t w) {
        return ((float)(w & 0x7fffffu) + 0.5f) * (1.0f / 8388608.0f);
    }
    __device__ __forceinline__ static float bridge_u(uint32_t wa, uint32_t wb) {
        return ((float)(((wa >> 23) << 9) | (wb >> 23)) + 0.5f) * (1.0f / 262144.0f);
    }

    // the walk ends at step nk (its steps before the exiting one: nk)
    __device__ __forceinline__ void exit_at(const ModelDev &M, ExitInfo<float> &ei, float ex, float ez,
                                            float th, int wall, uint32_t nk) {
        flush();
        ei.x = ex;
        ei.z = ez;
        ei.th = th;
        ei.wall = wall;
        ei.mlast = i;
        ei.nocc = nk;
        ei.aux = hits;
    }

    // A step that needs the long path (the position before it, its proposed
    // point and Philox words), and a step that hit an interface (hit
    // fraction, interface, side beyond it).  Both wait until the end of the iteration, where every lane of the
    // warp that has one runs it together: the per-step code stays short.
    float pX, pZ, pXn, pZn, pth, pxg;
    uint32_t pwa, pwb;
    int pside;

    // The long path of step n + k: the exact decisions of WalkerTM.
    // 0 no event, 1 exited, 2 interface hit (pending).
    __device__ __forceinline__ int rare(const ModelDev &M, const WalkArgs &A, float Xn, float Zn, uint32_t wa,
                                        uint32_t wb, uint32_t k, ExitInfo<float> &ei) {
        const uint32_t nk = n + k;
        if (nk == 0 && start_on_if) {
            flush();
            enter(M, A, i - 1);
            pXn = X;
            pZn = Z;
            pth = 0.f;
            pside = i + 1;
            pxg = X;
            return 2;
        }
        const float d[4] = {X + M.fhw, M.fhw - X, Z + M.fhh, M.fhh - Z};
        const float e[4] = {Xn + M.fhw, M.fhw - Xn, Zn + M.fhh, M.fhh - Zn};
        if (e[0] <= 0.f || e[1] <= 0.f || e[2] <= 0.f || e[3] <= 0.f) {
            float best = 3.f;
            int bw = 0;
#pragma unroll
            for (int w = 0; w < 4; ++w)
                if (e[w] <= 0.f) {
                    const float t = d[w] / (d[w] - e[w]);
                    if (t < best) { best = t; bw = w; }
                }
            place(M, Xn, Zn, best, bw, nk, ei);
            return 1;
        }
        // 2 d d' / (D_i dt) as c2 d d' (c2 = 2 / (D_i dt) of the strip)
        float best = 0.f;
        int bw = -1;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const float q = c2 * d[w] * e[w];
            if (bw < 0 || q < best) { best = q; bw = w; }
        }
        const float U = bridge_u(wa, wb);
        const float pw = best <= 40.f ? __expf(-best) : 0.f;
        if (U <= pw) {
            place(M, Xn, Zn, best / -__logf(U), bw, nk, ei);
            return 1;
        }
        const int j = strip(M, Xn);
        if (j != i) {
            const int jn = j > i ? i + 1 : i - 1;
            const float xi = j > i ? xr : xl;
            if (M.fdiff[jn] != Di) {
                flush();
                pXn = Xn;
                pZn = Zn;
                pth = fabsf((X - xi) / (Xn - X));
                pside = jn;
                pxg = xi;
                return 2;
            }
            // no regime change: the step's time goes to the strip of beta'
            flush();
            X = Xn;
            enter(M, A, j);
        } else {
            float bq = 0.f, bx = 0.f;
            int bs = -1;
            if (i > 0 && M.fdiff[i - 1] != Di) {
                bq = c2 * (X - xl) * (Xn - xl);
                bs = i - 1;
                bx = xl;
            }
            if (i < M.K - 1 && M.fdiff[i + 1] != Di) {
                const float q = c2 * (xr - X) * (xr - Xn);
                if (bs < 0 || q < bq) { bq = q; bs = i + 1; bx = xr; }
            }
            const float pg = (bs >= 0 && bq <= 40.f) ? __expf(-bq) : 0.f;
            if (pg > 0.f && U <= pw + (1.f - pw) * pg) {
                flush();
                pXn = Xn;
                pZn = Zn;
                pth = bq / -__logf((U - pw) / (1.f - pw));
                pside = bs;
                pxg = bx;
                return 2;
            }
        }
        run += 1;
        X = Xn;
        Z = Zn;
        dmin = fminf(M.fhw - fabsf(X), M.fhh - fabsf(Z));
        dI = fminf(X - xl, xr - X);
        return 0;
    }

    // The randomisation of a pending hit of step nk (crossing probability,
    // disc point, time split).  Returns true when the resampled point left
    // the domain (the walk ends on the nearest wall).
    __device__ __forceinline__ bool event(const ModelDev &M, const WalkArgs &A, uint32_t nk, ExitInfo<float> &ei) {
        // counter (nk, path, node id, 2): words 1 and 2 are the walk's, so the
        // first round's product of word 2 is the precomputed one of the steps
        const uint4 v = philox_rk_pre(nk, 2u, pre_x, pre_y, A.rk0, A.rk1);
        const float Dj = M.fdiff[pside];
        const float pi_ = Di / (Di + Dj), pj = Dj / (Di + Dj);
        const float zg = Z + pth * (pZn - Z);
        const float hh = sqrtf((float)A.dt * (Di > Dj ? Di : Dj));
        const float c = X <= pxg ? hh : -hh;
        const float rest = 1.f - pth;
        float cx;
        if (uni(v.y) < pi_) {
            h[32 * i] += 1.f - 0.5f * rest * pi_;
            h[32 * pside] += 0.5f * rest * pi_;
            cx = pxg - c;
        } else {
            const float ti = pth + 0.5f * rest * pj;
            h[32 * i] += ti;
            h[32 * pside] += 1.f - ti;
            cx = pxg + c;
        }
        float sa, ca;
        __sincosf(6.28318530718f * uni(v.w), &sa, &ca);
        const float rho = hh * sqrtf(uni(v.z));
        const float Xn = cx + rho * ca;
        const float Zn = zg + rho * sa;
        hits += 1;
        const float e[4] = {Xn + M.fhw, M.fhw - Xn, Zn + M.fhh, M.fhh - Zn};
        int bw = -1;
        float most = 0.f;
#pragma unroll
        for (int w = 0; w < 4; ++w)
            if (e[w] <= most && (bw < 0 || e[w] < most)) { most = e[w]; bw = w; }
        if (bw >= 0) {
            float ex = fminf(fmaxf(Xn, -M.fhw), M.fhw), ez = fminf(fmaxf(Zn, -M.fhh), M.fhh);
            if (bw == 0) ex = -M.fhw;
            if (bw == 1) ex = M.fhw;
            if (bw == 2) ez = -M.fhh;
            if (bw == 3) ez = M.fhh;
            exit_at(M, ei, ex, ez, 0.f, bw, nk);
            return true;
        }
        X = Xn;
        Z = Zn;
        dmin = fminf(M.fhw - fabsf(X), M.fhh - fabsf(Z));
        enter(M, A, strip(M, X));
        return false;
    }

    __device__ __forceinline__ void place(const ModelDev &M, float Xn, float Zn, float th, int w, uint32_t nk,
                                          ExitInfo<float> &ei) {
        float ex = fmaf(th, Xn - X, X), ez = fmaf(th, Zn - Z, Z);
        if (w == 0) ex = -M.fhw;
        if (w == 1) ex = M.fhw;
        if (w == 2) ez = -M.fhh;
        if (w == 3) ez = M.fhh;
        exit_at(M, ei, ex, ez, th, w, nk);
    }

    // (w mod 2^23 + 1/2) 2^-23 as the low 23 bits of w in the mantissa of a
    // float in [1, 2), minus 1 - 2^-24 (exact): the value of uni(w)
    __device__ __forceinline__ static float uni_m(uint32_t w) {
        return mant_one(w) - 0.99999994039535522f;
    }
    // One step of the short path, taken by every lane of the warp together
    // and always committed: the position moves to beta' whatever the lane's
    // state, so the unrolled steps need no branch around them and no copies
    // of the state.  The lane's first step that needs the long path (stop < 0
    // so far; not a skipped step, live false) records itself: its index k,
    // the position before it, its proposed point and its Philox words.  The
    // steps after it only move a position that iterate() then replaces by
    // the recorded one.  first: the walk's step 0 from a start on an
    // interface (a hit at t = 0).
    __device__ __forceinline__ void step(const ModelDev &M, const WalkArgs &A, uint32_t wa, uint32_t wb, int k,
                                         bool live, bool first, int &stop) {
        float sn, cs;
        // r = sqrt(-2 ln(u0) D_i dt) as sqrt(lc log2(u0)); |.| only guards the
        // last-ulp sign of lg2 near u0 = 1
        const float r = sqrtf(fabsf(lc * __log2f(uni_m(wa))));
        __sincosf(6.28318530718f * uni_m(wb), &sn, &cs);
        const float Xn = fmaf(r, cs, X);
        const float Zn = fmaf(r, sn, Z);
        const float dn = fminf(M.fhw - fabsf(Xn), M.fhh - fabsf(Zn));
        const float dIn = fminf(Xn - xl, xr - Xn);
        const float pn = dmin * dn, pI = dI * dIn;
        if (pn <= wthr || pI <= wthr || first) {
            // exact reject: every wall product is >= pn and every bound's
            // product >= pI, so p_w + p_g <= exp(-c2 pn) + exp(-c2 pI)
            if (stop < 0 && live && (first || bridge_u(wa, wb) <= __expf(-c2 * pn) + __expf(-c2 * pI))) {
                stop = k;
                pX = X;
                pZ = Z;
                pXn = Xn;
                pZn = Zn;
                pwa = wa;
                pwb = wb;
            }
        }
        X = live ? Xn : X;
        Z = live ? Zn : Z;
        dmin = live ? dn : dmin;
        dI = live ? dIn : dI;
    }

    // The steps of ROUNDS x PAIRS Philox calls, up to the lane's first step
    // that needs the long path; then the long path and the interface events
    // of the warp's lanes, once.  The rounds share the code of one (a loop,
    // not unrolled); more steps per long-path pass let more of the warp's
    // lanes have an event to resolve in it (measured on the analytic test
    // model with committed steps: 2, 4, 8 rounds -> 2.10, 2.25, 2.18e11
    // walk-steps/s; with the earlier layout, whose steps were each guarded
    // by the lane's state, 1, 2, 4 rounds -> 1.67, 1.79, 1.86e11).  A walk
    // within one iteration of max_steps takes its steps one at a time.
    // 0 running, 1 exited, 2 truncated.
    static constexpr int ROUNDS = 4;
    __device__ __forceinline__ int iterate(const ModelDev &M, const WalkArgs &A, uint32_t, ExitInfo<float> &ei) {
        const uint32_t odd = n & 1u;
        const uint32_t full = 2u * PAIRS * ROUNDS - odd;
        const bool first0 = n == 0 && start_on_if;
        int stop = -1;
        uint32_t done;
        if (A.max_steps - n >= full) {
#pragma unroll 1
            for (int r = 0; r < ROUNDS; ++r) {
                uint4 w[PAIRS];
#pragma unroll
                for (int q = 0; q < PAIRS; ++q)
                    w[q] = philox_rk_pre((n >> 1) + PAIRS * r + q, 0u, pre_x, pre_y, A.rk0, A.rk1);
                // k = steps of this walk since n; for an odd n the first word
                // pair of round 0 belongs to step n - 1 and is skipped
                const int kb = 2 * PAIRS * r - (int)odd;
#pragma unroll
                for (int q = 0; q < PAIRS; ++q) {
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const bool lead = q == 0 && hh == 0;
                        step(M, A, hh ? w[q].z : w[q].x, hh ? w[q].w : w[q].y, kb + 2 * q + hh,
                             lead ? (r != 0 || odd == 0u) : true, lead && r == 0 && first0, stop);
                    }
                }
            }
            done = stop >= 0 ? (uint32_t)stop + 1u : full;
        } else {
            const uint32_t lim = A.max_steps - n;
            for (uint32_t k = 0; k < lim && stop < 0; ++k) {
                const uint32_t sk = n + k;
                const uint4 w = philox_rk_pre(sk >> 1, 0u, pre_x, pre_y, A.rk0, A.rk1);
                step(M, A, (sk & 1u) ? w.z : w.x, (sk & 1u) ? w.w : w.y, (int)k, true, k == 0 && first0, stop);
            }
            done = stop >= 0 ? (uint32_t)stop + 1u : lim;
        }
        int st = 0;
        if (stop >= 0) {
            // back to the position before the recorded step; the steps before
            // it were spent in the current strip
            X = pX;
            Z = pZ;
            run += (uint32_t)stop;
            st = rare(M, A, pXn, pZn, pwa, pwb, (uint32_t)stop, ei);
        } else {
            run += done;
        }
        if (st == 1) return 1;
        if (st == 2 && event(M, A, n + done - 1, ei)) return 1;
        n += done;
        if (n >= A.max_steps) {
            exit_at(M, ei, X, Z, 0.f, 0, 0);
            ei.nocc = n;
            return 2;
        }
        return 0;
    }

    __device__ static void to_abs(const ModelDev &M, float Xc, float Zc, double &x, double &z) {
        x = (double)Xc + M.xc;
        z = (double)Zc + M.zc;
    }

    // The sample in single precision past the phase (FP64 is slow on this
    // GPU): the phase sum in FP64, reduced mod 2 pi, then FP32 functions.
    __device__ static double2 sample(const ModelDev &M, const SharedTables &T, const WalkArgs &A, int,
                                     int e, float xe, float ze, float th, int, int mlast, const Occ *c) {
        const double dt = A.dt;
        const double *kap = T.kappa + e * M.K;
        double ph = 0.0;
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
            if (k < M.K) ph = fma(kap[k], (double)c[k], ph);
        ph = fma(kap[mlast], (double)th, ph);
        ph *= 0.5 * dt;
        const double q = rint(ph * 0.15915494309189535);
        float sw, cw;
        __sincosf((float)fma(-q, 6.283185307179586, ph), &sw, &cw);
        const float x = xe + M.fxc, z = ze + M.fzc;
        float gr, gi;
        if (M.g_kind == 1) {
            const double *a = M.g_coef;
            gr = (float)(a[0] + a[2] * (double)x + a[4] * (double)z);
            gi = (float)(a[1] + a[3] * (double)x + a[5] * (double)z);
        } else if (M.g_kind == 2) {
            gr = x * x - z * z;
            gi = 0.f;
        } else if (M.g_kind == 3) {
            int s = 0;
            while (s < M.K - 1 && x >= M.fxif[s]) ++s;
            const float p = (float)M.tm_a[e][s][0] * x, qq = (float)M.tm_a[e][s][1] * x;
            float sq, cq;
            sincosf(qq, &sq, &cq);
            const float ep = expf(p), em = expf(-p);
            gr = (z + 1.f) * (0.5f * (ep + em) * cq);
            gi = (z + 1.f) * (0.5f * (ep - em) * sq);
        } else {
            float u = 0.f, a = (float)M.xmin;
            gr = 0.f;
            for (int k = 0; k < M.K; ++k) {
                const float b = k < M.K - 1 ? M.fxif[k] : (float)M.xmax;
                if (x <= b) {
                    gr = u + (x - a) / M.fdiff[k];
                    break;
                }
                u += (b - a) / M.fdiff[k];
                a = b;
                gr = u;
            }
            gi = 0.f;
        }
        return make_double2((double)(cw * gr + sw * gi), (double)(cw * gi - sw * gr));
    }
};

}  // namespace sdd
