// Single-precision walk (the throughput path).
//
// Position stepping, wall tests, material lookup and the per-walk phase
// factor are FP32; the per-material step counts are integers; the phase sum
// and the Monte Carlo sums are FP64.  Compiled with -ftz=true
// -prec-div=false -prec-sqrt=false.
//
// One Euler-Maruyama step of Sec. 3.1 (discretised process, kappa_i = 1):
//   (u0, u1)  two uniforms (w mod 2^23 + 1/2) 2^-23 from one Philox call,
//   r^2 = -2 ln(u0) dt,  beta' = beta + r (cos 2 pi u1, sin 2 pi u1),
// then the boundary rule of the first-exit-time estimate: overshoot ->
// theta = d / (d + |d'|) on the first wall reached; else the Brownian-bridge
// test 2 d d' / dt <= -ln U_gamma with one uniform per step (18 spare bits of
// the step's Philox words); else the step's time goes to the material of
// beta' (Sec. 3.1, no regime change for TE).
//
// The walk runs in centred coordinates X = x - xc, Z = z - zc, so the
// distance to the nearer wall of each pair is h - |X|.  Two steps share one
// Philox call (words 0,1 for the even step, 2,3 for the odd one), and one
// call of iterate() runs 8 steps (4 with 8 materials).
#include <type_traits>

#include "walk_sched.cuh"
#include "walk_tm.cuh"

namespace sdd {

// Uniforms of the single-precision walk: the low 23 bits of a Philox word as
// the mantissa of a float in [1, 2); u = (w mod 2^23 + 1/2) 2^-23 exactly
// (1.m - (1 - 2^-24), an exact difference by Sterbenz' lemma).
__device__ __forceinline__ float one_plus(uint32_t w) { return mant_one(w); }
__device__ __forceinline__ float uni23(uint32_t w) { return one_plus(w) - 0.99999994039535522f; }

// Occupation counters.  KMAX = 2: the step count of material 1.  KMAX = 3, 4:
// power sums s_p = sum over steps of m^p (p = 1 .. KMAX-1), which determine
// the counts of materials 1 .. KMAX-1 (a Vandermonde system, solved once at
// the exit).  KMAX = 8: a per-lane histogram in shared memory, one shared
// atomic add per step.
template <int KMAX>
struct Occupancy {
    uint32_t s[KMAX > 1 ? KMAX - 1 : 1];
    __device__ __forceinline__ void bind(uint32_t) {}
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int j = 0; j < (KMAX > 1 ? KMAX - 1 : 1); ++j) s[j] = 0;
    }
    __device__ __forceinline__ void add(int m) {
        const uint32_t u = (uint32_t)m;
        if (KMAX == 2) {
            s[0] += u;
        } else if (KMAX == 3) {
            s[0] += u;
            s[1] += u * u;
        } else if (KMAX == 4) {
            const uint32_t u2 = u * u;
            s[0] += u;
            s[1] += u2;
            s[2] += u2 * u;
        } else {
#pragma unroll
            for (int j = 1; j < KMAX; ++j) s[j - 1] += (m == j) ? 1u : 0u;
        }
    }
    // counts of materials 1 .. KMAX-1
    __device__ __forceinline__ void counts(uint32_t *c) const {
        if (KMAX == 2) {
            c[0] = s[0];
        } else if (KMAX == 3) {
            // s1 = c1 + 2 c2, s2 = c1 + 4 c2
            const uint32_t c2 = (s[1] - s[0]) >> 1;
            c[1] = c2;
            c[0] = s[0] - 2u * c2;
        } else if (KMAX == 4) {
            // s1 = c1 + 2 c2 + 3 c3, s2 = c1 + 4 c2 + 9 c3, s3 = c1 + 8 c2 + 27 c3
            const uint32_t c3 = (s[2] - 3u * s[1] + 2u * s[0]) / 6u;
            const uint32_t c2 = (s[1] - s[0] - 6u * c3) >> 1;
            c[2] = c3;
            c[1] = c2;
            c[0] = s[0] - 2u * c2 - 3u * c3;
        } else {
#pragma unroll
            for (int j = 0; j < KMAX - 1; ++j) c[j] = s[j];
        }
    }
};

template <>
struct Occupancy<8> {
    uint32_t base;  // shared address of hist[0][lane]; material m at base + 128 m
    __device__ __forceinline__ void bind(uint32_t a) { base = a; }
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int j = 0; j < 8; ++j) asm volatile("st.shared.u32 [%0], %1;" ::"r"(base + 128u * j), "r"(0u));
    }
    __device__ __forceinline__ void add(int m) {
        asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(base + ((uint32_t)m << 7)), "r"(1u));
    }
    __device__ __forceinline__ void counts(uint32_t *c) const {
#pragma unroll
        for (int j = 1; j < 8; ++j) {
            uint32_t v;
            asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(base + 128u * j));
            c[j - 1] = v;
        }
    }
};

// Region counters of the one-shape programs (GC_CONTACT, GC_RECT1, GC_TRI1): ce steps
// on the earth side of the surface, cs steps inside the shape.  The shape
// lies wholly on one side of the surface, so these two give every
// material's count at the exit (WalkerF32::counts).
struct Regions {
    uint32_t ce, cs;
    __device__ __forceinline__ void bind(uint32_t) {}
    __device__ __forceinline__ void clear() { ce = 0u; cs = 0u; }
};

// GC: the material-lookup program (GeoCode).  Shape parameters are read
// with compile-time indices, so every one is an immediate constant operand.
template <int KMAX_, int GC>
struct WalkerF32 {
    using Real = float;
    static constexpr int KMAX = KMAX_;
    // records: step counts of materials 1..K-1 (material 0 from the total)
    using Occ = uint32_t;
    using HistT = uint32_t;
    static constexpr int kStored = KMAX - 1;
    static constexpr int kHist = KMAX == 8 ? 8 : 1;
    static constexpr bool kGrouped = GC == GC_RASTER_MULTI;
    // 24 resident warps whose iterations carry four independent Philox
    // chains keep the issue slots fuller than 32 warps in 64 registers
    static constexpr int kMinCTAs = 3;

    // one-shape programs count regions (two predicated adds per step in
    // place of the material selects and the power sums)
    static constexpr bool kRegions = GC == GC_CONTACT || GC == GC_RECT1 || GC == GC_TRI1;

    float X, Z, dmin;  // centred position, distance to the nearest wall
    uint32_t n;        // Euler steps accepted (even at the start of iterate)
    typename std::conditional<kRegions, Regions, Occupancy<KMAX>>::type occ;
    uint32_t nid, pre_x, pre_y;
    const uint32_t *tco;  // GC_RASTER_MULTI: the tile map of this walk's model

    __device__ __forceinline__ static bool in_rect(const ShapeDev &S, float X, float Z) {
        return X >= S.f[0] && X < S.f[1] && Z >= S.f[2] && Z < S.f[3];
    }
    __device__ __forceinline__ static bool in_tri(const ShapeDev &S, float X, float Z) {
        return fmaf(S.f[0], X, fmaf(S.f[1], Z, S.f[2])) >= 0.f &&
               fmaf(S.f[3], X, fmaf(S.f[4], Z, S.f[5])) >= 0.f &&
               fmaf(S.f[6], X, fmaf(S.f[7], Z, S.f[8])) >= 0.f;
    }

    __device__ __forceinline__ int material(const ModelDev &M, float X, float Z) const {
        if (GC == GC_RASTER || GC == GC_RASTER_MULTI) {
            // round(v - 1/2) = floor(v) for v = (X + hw) sx >= 0 (magic-number
            // rounding), plus kTile: the index into the tile map, which starts
            // one tile before the raster.  A point inside the domain gives a cell
            // index in -1 .. n (rounding can reach one past an edge), and the
            // map's margin tiles repeat the edge cells, so no clamp is needed.
            // Two-level lookup: the coarse entry (L1-resident) is the material
            // of a uniform tile, else the tile's cells in the pool.
            const int ix = __float_as_int(fmaf(X, M.fsx, M.fox) + 12582912.0f) - 0x4B400000;
            const int iz = __float_as_int(fmaf(Z, M.fsz, M.foz) + 12582912.0f) - 0x4B400000;
            const uint32_t *co = GC == GC_RASTER_MULTI ? tco : M.tcoarse;
            const uint32_t c = __ldg(co + (iz >> kTileShift) * M.ntx + (ix >> kTileShift));
            if (c & kTileUniform) return (int)(c & 0xffu);
            const uint8_t *po = reinterpret_cast<const uint8_t *>(co) + M.tpool_off;
            return (int)__ldg(po + ((size_t)c << (2 * kTileShift)) + ((iz & (kTile - 1)) << kTileShift) +
                              (ix & (kTile - 1)));
        }
        const int m = (Z >= M.fzs) ? M.bg_earth : M.bg_air;
        if (GC == GC_LAYER) return m;
        if (GC == GC_RECT1) return in_rect(M.shapes[0], X, Z) ? M.shapes[0].mat : m;
        if (GC == GC_CONTACT) return (Z >= M.fzs && X >= M.shapes[0].f[0]) ? M.shapes[0].mat : m;
        if (GC == GC_TRI1) return in_tri(M.shapes[0], X, Z) ? M.shapes[0].mat : m;
        constexpr int NS = GC == GC_SHAPES4 ? 4 : kMaxShapes;
        int r = m;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            if (s < M.n_shapes) {
                const ShapeDev &S = M.shapes[s];
                const bool in = S.kind == 0 ? in_rect(S, X, Z) : in_tri(S, X, Z);
                r = in ? S.mat : r;
            }
        }
        return r;
    }

    // The step at (X, Z) into the region counters: the earth test and the
    // shape test of material() as predicates, each adding one to its counter
    // (compares with .ftz, as the unit's float compares).
    __device__ __forceinline__ void count_regions(const ModelDev &M, float X, float Z) {
        if (GC == GC_CONTACT) {
            asm("{\n\t.reg .pred pe, ps;\n\t"
                "setp.ge.ftz.f32 pe, %3, %4;\n\t"
                "setp.ge.and.ftz.f32 ps, %2, %5, pe;\n\t"
                "@pe add.u32 %0, %0, 1;\n\t"
                "@ps add.u32 %1, %1, 1;\n\t}"
                : "+r"(occ.ce), "+r"(occ.cs)
                : "f"(X), "f"(Z), "f"(M.fzs), "f"(M.shapes[0].f[0]));
        } else if (GC == GC_TRI1) {
            // the three edge functions as in in_tri(), the compares chained
            const ShapeDev &S = M.shapes[0];
            const float e0 = fmaf(S.f[0], X, fmaf(S.f[1], Z, S.f[2]));
            const float e1 = fmaf(S.f[3], X, fmaf(S.f[4], Z, S.f[5]));
            const float e2 = fmaf(S.f[6], X, fmaf(S.f[7], Z, S.f[8]));
            asm("{\n\t.reg .pred pe, ps;\n\t"
                "setp.ge.ftz.f32 pe, %2, %3;\n\t"
                "setp.ge.ftz.f32 ps, %4, 0f00000000;\n\t"
                "setp.ge.and.ftz.f32 ps, %5, 0f00000000, ps;\n\t"
                "setp.ge.and.ftz.f32 ps, %6, 0f00000000, ps;\n\t"
                "@pe add.u32 %0, %0, 1;\n\t"
                "@ps add.u32 %1, %1, 1;\n\t}"
                : "+r"(occ.ce), "+r"(occ.cs)
                : "f"(Z), "f"(M.fzs), "f"(e0), "f"(e1), "f"(e2));
        } else {
            asm("{\n\t.reg .pred pe, ps;\n\t"
                "setp.ge.ftz.f32 pe, %3, %4;\n\t"
                "setp.ge.ftz.f32 ps, %2, %5;\n\t"
                "setp.lt.and.ftz.f32 ps, %2, %6, ps;\n\t"
                "setp.ge.and.ftz.f32 ps, %3, %7, ps;\n\t"
                "setp.lt.and.ftz.f32 ps, %3, %8, ps;\n\t"
                "@pe add.u32 %0, %0, 1;\n\t"
                "@ps add.u32 %1, %1, 1;\n\t}"
                : "+r"(occ.ce), "+r"(occ.cs)
                : "f"(X), "f"(Z), "f"(M.fzs), "f"(M.shapes[0].f[0]), "f"(M.shapes[0].f[1]),
                  "f"(M.shapes[0].f[2]), "f"(M.shapes[0].f[3]));
        }
    }

    // Counts of materials 1 .. KMAX-1 after nocc counted steps.  Region
    // counters: the shape has cs; with the shape in the earth the earth
    // background has ce - cs and the air nocc - ce, with the shape in the air
    // the earth has ce and the air nocc - ce - cs.
    __device__ __forceinline__ void counts(const ModelDev &M, uint32_t nocc, uint32_t *c) const {
        if constexpr (kRegions) {
            const uint32_t ce = occ.ce, cs = occ.cs;
            const uint32_t ear = M.shape_air ? ce : ce - cs;
            const uint32_t air = nocc - ce - (M.shape_air ? cs : 0u);
            const int ma = M.bg_air, me = M.bg_earth, msh = M.shapes[0].mat;
#pragma unroll
            for (int j = 1; j < KMAX; ++j)
                c[j - 1] = (ma == j ? air : 0u) + (me == j ? ear : 0u) + (msh == j ? cs : 0u);
        } else {
            occ.counts(c);
        }
    }
    __device__ __forceinline__ void bind(HistT *h) { occ.bind((uint32_t)__cvta_generic_to_shared(h)); }

    __device__ __forceinline__ void start(const ModelDev &M, const WalkArgs &A, double x0,
                                          double z0, uint32_t path, uint32_t node_id, int model) {
        if (GC == GC_RASTER_MULTI) tco = A.models[model].tcoarse;
        X = (float)(x0 - M.xc);
        Z = (float)(z0 - M.zc);
        dmin = fminf(M.fhw - fabsf(X), M.fhh - fabsf(Z));
        n = 0;
        occ.clear();
        nid = node_id;
        pre_x = __umulhi(0xCD9E8D57u, node_id) ^ path ^ A.rk0[0];
        pre_y = 0xCD9E8D57u * node_id;
    }

    __device__ __forceinline__ void place(const ModelDev &M, float Xn, float Zn, float th, int w,
                                          ExitInfo<float> &ei) const {
        ei.th = th;
        ei.wall = w;
        ei.x = fmaf(th, Xn - X, X);
        ei.z = fmaf(th, Zn - Z, Z);
        if (w == 0) ei.x = -M.fhw;
        if (w == 1) ei.x = M.fhw;
        if (w == 2) ei.z = -M.fhh;
        if (w == 3) ei.z = M.fhh;
        ei.mlast = material(M, X, Z);
    }

    // The step (X, Z) -> (Xn, Zn) came within reach of a wall (rare; taken by
    // few lanes of a warp at a time, so kept short).  Overshoot (dn <= 0):
    // theta_w = d_w / (d_w - d'_w) over the walls with d'_w <= 0, smallest
    // first, ties to the first of left, right, top, bottom.  Both inside: the
    // Brownian-bridge test with one uniform for all walls: the walk touched a
    // wall iff 2 d_w d'_w / dt <= -ln U for the smallest product, tested as
    // U <= exp(-2 d_w d'_w / dt).  U is made of the 18 bits of the step's two
    // Philox words that the normals leave unused:
    // U = (high 9 bits of wa : high 9 bits of wb + 1/2) 2^-18.  Every
    // product d_w d'_w is at least pn = dmin dn (the nearest distances before
    // and after the step), so U > exp(-2 pn / dt) rules out a hit without
    // forming the four products; most near-wall steps end there.
    __device__ __forceinline__ bool near_wall(const ModelDev &M, const WalkArgs &A, float Xn,
                                              float Zn, float dn, float pn, uint32_t wa, uint32_t wb,
                                              ExitInfo<float> &ei) const {
        const float d[4] = {X + M.fhw, M.fhw - X, Z + M.fhh, M.fhh - Z};
        const float e[4] = {Xn + M.fhw, M.fhw - Xn, Zn + M.fhh, M.fhh - Zn};
        const uint32_t u18 = ((wa >> 23) << 9) | (wb >> 23);
        const float U = fmaf((float)u18, 3.814697265625e-06f, 1.9073486328125e-06f);
        if (dn > 0.f && U > __expf(-pn * A.f_c2dt)) return false;
        if (dn <= 0.f) {
            float best = 2.0f;
            int bw = 0;
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                if (e[w] <= 0.f) {
                    const float t = d[w] / (d[w] - e[w]);
                    if (t < best) { best = t; bw = w; }
                }
            }
            place(M, Xn, Zn, best, bw, ei);
            return true;
        }
        const float p0 = d[0] * e[0], p1 = d[1] * e[1], p2 = d[2] * e[2], p3 = d[3] * e[3];
        const float pmin = fminf(fminf(p0, p1), fminf(p2, p3));
        const float es = pmin * A.f_c2dt;
        if (U > __expf(-es)) return false;
        // a hit: the wall of the smallest product (first in wall order) and
        // the fraction theta = (2 d d' / dt) / (-ln U)
        const int bw = p0 == pmin ? 0 : (p1 == pmin ? 1 : (p2 == pmin ? 2 : 3));
        place(M, Xn, Zn, es / -logf(U), bw, ei);
        return true;
    }

    // The part of an Euler step that does not depend on the position: the
    // step length r = sqrt(-2 ln(u0) dt) and direction of the normal pair
    // (angle 2 pi (u1 - 1/2), so cos(2 pi u1) = -cs and sin(2 pi u1) = -sn)
    // from the step's Philox words (wa, wb).
    struct Incr {
        float r, sn, cs;
    };
    __device__ __forceinline__ static Incr increment(const WalkArgs &A, uint32_t wa, uint32_t wb) {
        Incr d;
        // |.| only guards the last-ulp sign of lg2 near u0 = 1
        d.r = sqrtf(fabsf(A.f_cdt * __log2f(uni23(wa))));
        __sincosf(fmaf(one_plus(wb), 6.28318530718f, -9.42477796077f), &d.sn, &d.cs);
        return d;
    }

    // The rest of the step: move, test the walls, count the occupation.
    // Only the high 9 bits of wa and wb are read (the bridge uniform, on the
    // rare steps near a wall).  k = steps of this walk since n.  Returns true
    // when the walk reached the boundary.
    __device__ __forceinline__ bool advance(const ModelDev &M, const WalkArgs &A, const Incr &d,
                                            uint32_t wa, uint32_t wb, uint32_t k, ExitInfo<float> &ei) {
        const float Xn = fmaf(-d.r, d.cs, X);
        const float Zn = fmaf(-d.r, d.sn, Z);
        const float dn = fminf(M.fhw - fabsf(Xn), M.fhh - fabsf(Zn));
        const float pn = dmin * dn;
        if (pn <= A.f_bthr) {
            if (near_wall(M, A, Xn, Zn, dn, pn, wa, wb, ei)) {
                ei.nocc = n + k;
                return true;
            }
        }
        if constexpr (kRegions) count_regions(M, Xn, Zn);
        else occ.add(material(M, Xn, Zn));
        X = Xn;
        Z = Zn;
        dmin = dn;
        return false;
    }

    __device__ __forceinline__ bool substep(const ModelDev &M, const WalkArgs &A, uint32_t wa,
                                            uint32_t wb, uint32_t k, ExitInfo<float> &ei) {
        return advance(M, A, increment(A, wa, wb), wa, wb, k, ei);
    }

    // Raster programs with up to 8 materials: the walk does not depend on the
    // materials it crosses, so an iteration records each accepted step's
    // tile-map coordinates (the coarse index, and the cell's offset in its
    // tile, 4 to a word) and looks them up together after its steps, as
    // independent loads in flight at once instead of one dependent chain per
    // step (measured: +3 % on one 6-material raster, +7.6 % on a 12-model
    // batch; with K <= 4 the per-step lookup stays faster, 2.6e11 against
    // 1.7e11 walk-steps/s).
    static constexpr bool kDeferLookup = (GC == GC_RASTER || GC == GC_RASTER_MULTI) && KMAX == 8;

    __device__ __forceinline__ static void cell_of(const ModelDev &M, float X, float Z, uint32_t &ci,
                                                   uint32_t &off, int k) {
        const int ix = __float_as_int(fmaf(X, M.fsx, M.fox) + 12582912.0f) - 0x4B400000;
        const int iz = __float_as_int(fmaf(Z, M.fsz, M.foz) + 12582912.0f) - 0x4B400000;
        ci = (uint32_t)((iz >> kTileShift) * M.ntx + (ix >> kTileShift));
        const uint32_t o = (uint32_t)(((iz & (kTile - 1)) << kTileShift) | (ix & (kTile - 1)));
        off = (k & 3) == 0 ? o : off | (o << (8 * (k & 3)));
    }

    // The step of advance() with the material lookup deferred.
    __device__ __forceinline__ bool advance_cell(const ModelDev &M, const WalkArgs &A, const Incr &d,
                                                 uint32_t wa, uint32_t wb, uint32_t k, ExitInfo<float> &ei,
                                                 uint32_t &ci, uint32_t &off) {
        const float Xn = fmaf(-d.r, d.cs, X);
        const float Zn = fmaf(-d.r, d.sn, Z);
        const float dn = fminf(M.fhw - fabsf(Xn), M.fhh - fabsf(Zn));
        const float pn = dmin * dn;
        if (pn <= A.f_bthr) {
            if (near_wall(M, A, Xn, Zn, dn, pn, wa, wb, ei)) {
                ei.nocc = n + k;
                return true;
            }
        }
        cell_of(M, Xn, Zn, ci, off, (int)k);
        X = Xn;
        Z = Zn;
        dmin = dn;
        return false;
    }

    // Count the materials of the first cnt recorded steps: all coarse
    // entries first, then the cells of mixed tiles.
    template <int NS>
    __device__ __forceinline__ void add_cells(const ModelDev &M, const uint32_t (&ci)[NS],
                                              const uint32_t (&off)[(NS + 3) / 4], int cnt) {
        const uint32_t *co = GC == GC_RASTER_MULTI ? tco : M.tcoarse;
        const uint8_t *po = reinterpret_cast<const uint8_t *>(co) + M.tpool_off;
        uint32_t c[NS];
#pragma unroll
        for (int j = 0; j < NS; ++j) c[j] = j < cnt ? __ldg(co + ci[j]) : kTileUniform;
        int m[NS];
#pragma unroll
        for (int j = 0; j < NS; ++j) {
            const uint32_t o = (off[j >> 2] >> (8 * (j & 3))) & 0xffu;
            m[j] = (c[j] & kTileUniform) ? (int)(c[j] & 0xffu)
                                         : (int)__ldg(po + ((size_t)c[j] << (2 * kTileShift)) + o);
        }
#pragma unroll
        for (int j = 0; j < NS; ++j)
            if (j < cnt) occ.add(m[j]);
    }

    // PAIRS Philox calls, two Euler steps each, per call of iterate: the
    // per-iteration work of the scheduler loop (constants, vote, branch) is
    // shared by 2 PAIRS steps.  The calls depend only on the step counter, so
    // all of them are issued first, as independent chains the SM can overlap
    // (a walk that exits early discards the rest).  0 running, 1 exited,
    // 2 truncated (max_steps is a multiple of 8, so a walk is only truncated
    // at the end of an iteration).
    static constexpr int PAIRS = KMAX == 8 ? 2 : 4;

    __device__ __forceinline__ int iterate(const ModelDev &M, const WalkArgs &A, uint32_t path,
                                           ExitInfo<float> &ei) {
        uint4 w[PAIRS];
#pragma unroll
        for (int q = 0; q < PAIRS; ++q) w[q] = philox_rk_pre((n >> 1) + q, 0u, pre_x, pre_y, A.rk0, A.rk1);
        if constexpr (kDeferLookup) {
            constexpr int NS = 2 * PAIRS;
            uint32_t ci[NS], off[(NS + 3) / 4];
            int done = NS;
#pragma unroll
            for (int k = 0; k < NS; ++k) {
                if (done == NS) {
                    const uint32_t wa = (k & 1) ? w[k >> 1].z : w[k >> 1].x;
                    const uint32_t wb = (k & 1) ? w[k >> 1].w : w[k >> 1].y;
                    if (advance_cell(M, A, increment(A, wa, wb), wa, wb, (uint32_t)k, ei, ci[k], off[k >> 2]))
                        done = k;
                }
            }
            add_cells(M, ci, off, done);
            if (done < NS) return 1;
        } else {
#pragma unroll
            for (int q = 0; q < PAIRS; ++q) {
                if (substep(M, A, w[q].x, w[q].y, 2u * q, ei)) return 1;
                if (substep(M, A, w[q].z, w[q].w, 2u * q + 1u, ei)) return 1;
            }
        }
        n += 2 * PAIRS;
        if (n >= A.max_steps) {
            ei.x = X; ei.z = Z; ei.th = 0.f; ei.wall = 0;
            ei.mlast = material(M, X, Z);
            ei.nocc = n;
            return 2;
        }
        return 0;
    }

    // Cooperative tail (scheduler): once few walks are left, every lane of
    // the warp computes increments for them, and each walk then runs only
    // the position-dependent chain of its steps.  The increments are the
    // ones increment() gives in iterate(), so the walks are the same.
    static constexpr bool kCoop = true;
    __device__ __forceinline__ uint32_t steps() const { return n; }
    __device__ __forceinline__ uint2 key() const { return make_uint2(pre_x, pre_y); }

    // The two increments of Philox pair q of a walk with step counter n0
    // (even) and key (pre_x, pre_y); the fourth word keeps the high 9 bits of
    // wa (bits 31..23) and of wb (bits 22..14).
    __device__ __forceinline__ static void pair_increments(const WalkArgs &A, uint32_t n0, uint2 key,
                                                           uint32_t q, float4 &s0, float4 &s1) {
        const uint4 w = philox_rk_pre((n0 >> 1) + q, 0u, key.x, key.y, A.rk0, A.rk1);
        const Incr a = increment(A, w.x, w.y), b = increment(A, w.z, w.w);
        s0 = make_float4(a.r, a.sn, a.cs, __uint_as_float((w.x & 0xff800000u) | (w.y >> 9)));
        s1 = make_float4(b.r, b.sn, b.cs, __uint_as_float((w.z & 0xff800000u) | (w.w >> 9)));
    }

    // Steps with the cnt (even) increments d[0 .. cnt-1].  0 running,
    // 1 exited, 2 truncated (at max_steps exactly, as in iterate()).
    __device__ __forceinline__ int consume(const ModelDev &M, const WalkArgs &A, const float4 *d,
                                           int cnt, ExitInfo<float> &ei) {
        for (int k = 0; k < cnt; ++k) {
            const float4 v = d[k];
            Incr c;
            c.r = v.x;
            c.sn = v.y;
            c.cs = v.z;
            const uint32_t hb = __float_as_uint(v.w);
            if (advance(M, A, c, hb & 0xff800000u, hb << 9, (uint32_t)k, ei)) return 1;
            if (n + (uint32_t)k + 1u >= A.max_steps) {
                n += (uint32_t)k + 1u;
                ei.x = X; ei.z = Z; ei.th = 0.f; ei.wall = 0;
                ei.mlast = material(M, X, Z);
                ei.nocc = n;
                return 2;
            }
        }
        n += (uint32_t)cnt;
        return 0;
    }

    __device__ static void to_abs(const ModelDev &M, float X, float Z, double &x, double &z) {
        x = (double)X + M.xc;
        z = (double)Z + M.zc;
    }

    // 1D column solution at depth z: exp(-k z) in the earth, 1 - k z in air.
    __device__ static void column(float kr, float ki, float z, float &gr, float &gi) {
        if (z >= 0.f) {
            const float a = expf(-kr * z);
            float s, c;
            sincosf(ki * z, &s, &c);
            gr = a * c;
            gi = -a * s;
        } else {
            gr = fmaf(-kr, z, 1.f);
            gi = -ki * z;
        }
    }

    // Sample of one walk for evaluation e: g(exit) exp(-i (1/2) sum_m kappa_{e,m} T_m).
    __device__ static double2 sample(const ModelDev &M, const SharedTables &T, const WalkArgs &A,
                                     int model, int e, float X, float Z, float th, int wall,
                                     int mlast, const uint32_t *c) {
        const double dt = A.dt;
        const bool multi = GC == GC_RASTER_MULTI;
        const int K = multi ? A.models[model].K : M.K;
        const double *kap = (multi ? A.models[model].kappa : T.kappa) + e * K;
        double ph = 0.0;
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
            if (k < K) ph = fma(kap[k], (double)c[k], ph);
        ph = fma(kap[mlast], (double)th, ph);
        ph *= 0.5 * dt;
        const double q = rint(ph * 0.15915494309189535);
        const float pr = (float)fma(-q, 6.283185307179586, ph);
        float sw, cw;
        sincosf(pr, &sw, &cw);
        float gr, gi;
        const float x = X + M.fxc, z = Z + M.fzc;
        if (M.g_kind == 1) {
            const double *a = M.g_coef;
            gr = (float)(a[0] + a[2] * (double)x + a[4] * (double)z);
            gi = (float)(a[1] + a[3] * (double)x + a[5] * (double)z);
        } else if (M.g_kind == 2) {
            gr = x * x - z * z;
            gi = 0.f;
        } else {
            const EvalDev &E = multi ? A.models[model].ev[e] : T.ev[e];
            if (wall == 0) {
                column((float)E.kl_re, (float)E.kl_im, z, gr, gi);
            } else if (wall == 1) {
                column((float)E.kr_re, (float)E.kr_im, z, gr, gi);
            } else {
                const float t = (X + M.fhw) / (2.f * M.fhw);
                const double lr = wall == 2 ? E.tl_re : E.bl_re, li = wall == 2 ? E.tl_im : E.bl_im;
                const double rr = wall == 2 ? E.tr_re : E.br_re, ri = wall == 2 ? E.tr_im : E.br_im;
                gr = fmaf(t, (float)(rr - lr), (float)lr);
                gi = fmaf(t, (float)(ri - li), (float)li);
            }
        }
        // (cw - i sw)(gr + i gi)
        return make_double2((double)fmaf(cw, gr, sw * gi), (double)fmaf(cw, gi, -sw * gr));
    }
};

template <int KMAX, int GC>
static cudaError_t launch_one(const ModelDev &M, const WalkArgs &A, int grid, int block,
                              cudaStream_t s) {
    const size_t sm = shared_bytes<WalkerF32<KMAX, GC>>(block / 32, M.E, M.K);
    auto k = walk_kernel<WalkerF32<KMAX, GC>>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k<<<grid, block, sm, s>>>(M, A);
    return cudaGetLastError();
}

template <int KMAX, int GC>
static int occ_one(int block, int E, int K) {
    const size_t sm = shared_bytes<WalkerF32<KMAX, GC>>(block / 32, E, K);
    auto k = walk_kernel<WalkerF32<KMAX, GC>>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, sm) != cudaSuccess) return 0;
    return n;
}

// Kernel variants: materials K <= KMAX in {2, 3, 4, 8} x the six lookup programs.
#define SDD_GC_CASES(FN, KM, ...)                                               \
    switch (gcode) {                                                            \
    case GC_LAYER: return FN<KM, GC_LAYER>(__VA_ARGS__);                        \
    case GC_RECT1: return FN<KM, GC_RECT1>(__VA_ARGS__);                        \
    case GC_TRI1: return FN<KM, GC_TRI1>(__VA_ARGS__);                          \
    case GC_SHAPES4: return FN<KM, GC_SHAPES4>(__VA_ARGS__);                    \
    case GC_SHAPES16: return FN<KM, GC_SHAPES16>(__VA_ARGS__);                  \
    case GC_RASTER: return FN<KM, GC_RASTER>(__VA_ARGS__);                      \
    case GC_CONTACT: return FN<KM, GC_CONTACT>(__VA_ARGS__);                    \
    case GC_RASTER_MULTI: return FN<KM, GC_RASTER_MULTI>(__VA_ARGS__);          \
    default: break;                                                             \
    }

#define SDD_DISPATCH(FN, ...)                                                   \
    switch (kmax) {                                                             \
    case 2: SDD_GC_CASES(FN, 2, __VA_ARGS__) break;                             \
    case 3: SDD_GC_CASES(FN, 3, __VA_ARGS__) break;                             \
    case 4: SDD_GC_CASES(FN, 4, __VA_ARGS__) break;                             \
    case 8: SDD_GC_CASES(FN, 8, __VA_ARGS__) break;                             \
    default: break;                                                             \
    }

// The TM walk (vertical strips, K <= KMAX in {2, 3, 4, 8}).
template <int KMAX>
static cudaError_t launch_tm(const ModelDev &M, const WalkArgs &A, int grid, int block, cudaStream_t s) {
    using W = WalkerTM32<KMAX>;
    const size_t sm = shared_bytes<W>(block / 32, M.E, M.K);
    auto k = walk_kernel<W>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k<<<grid, block, sm, s>>>(M, A);
    return cudaGetLastError();
}

template <int KMAX>
static int occ_tm(int block, int E, int K) {
    using W = WalkerTM32<KMAX>;
    const size_t sm = shared_bytes<W>(block / 32, E, K);
    auto k = walk_kernel<W>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, sm) != cudaSuccess) return 0;
    return n;
}

#define SDD_TM_DISPATCH(FN, ...)                                                \
    switch (kmax) {                                                             \
    case 2: return FN<2>(__VA_ARGS__);                                          \
    case 3: return FN<3>(__VA_ARGS__);                                          \
    case 4: return FN<4>(__VA_ARGS__);                                          \
    case 8: return FN<8>(__VA_ARGS__);                                          \
    default: break;                                                             \
    }

cudaError_t launch_walk_f32(int kmax, int /*geo*/, const ModelDev &M, const WalkArgs &A, int grid,
                            int block, cudaStream_t s) {
    const int gcode = M.gcode;
    if (gcode == GC_TM) {
        SDD_TM_DISPATCH(launch_tm, M, A, grid, block, s)
        return cudaErrorInvalidValue;
    }
    SDD_DISPATCH(launch_one, M, A, grid, block, s)
    return cudaErrorInvalidValue;
}

int occupancy_f32(int kmax, int gcode, int block, int E, int K) {
    if (gcode == GC_TM) {
        SDD_TM_DISPATCH(occ_tm, block, E, K)
        return 0;
    }
    SDD_DISPATCH(occ_one, block, E, K)
    return 0;
}

}  // namespace sdd
