// Persistent walk scheduler shared by the single- and double-precision walks.
//
// Work model.  The estimator of Sec. 3.1 averages independent walks per
// interface node; the node values are independent of one another (Sec. 5).
// The host cuts every node's paths into work items (node, path range) and
// orders them so that item sizes shrink toward the end of the queue (guided
// self-scheduling, down to one walk per lane): when the queue runs dry, every
// warp holds little unfinished work.  Each warp of a persistent grid takes
// items from a global atomic counter and keeps its 32 lanes busy: a lane
// whose walk has reached the boundary takes the next path of the warp's
// current item at once, and the warp opens the next item as soon as the
// current one is fully handed out, however many earlier items still have
// walks in flight.  Uneven exit times therefore idle no lane until the queue
// is empty.
//
// Exit records.  A finished walk writes a small record (item, exit point,
// hit fraction theta, wall, last material, per-material step counts) into a
// per-warp ring in shared memory.  Once 32 records are waiting, the whole
// warp turns them into samples g(exit) exp(-i (1/2) sum_m kappa_{e,m} T_m)
// for every evaluation e, lane l handling evaluation l mod Epad.  The samples
// of each item are summed across the lanes with warp shuffles (fixed order)
// and lane e adds them to the item's slot in global memory (sum re, sum im,
// sum re^2, sum im^2; a few MB, L2-resident).  An item belongs to the one
// warp that opened it, so its slot needs no atomics.  A second kernel adds
// the slots of each node in item order.
#pragma once

#include "sdd_internal.cuh"

namespace sdd {

constexpr unsigned kFull = 0xffffffffu;

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit products with multipliers 0xD2511F53 and 0xCD9E8D57, the
// key bumped by 0x9E3779B9 / 0xBB67AE85 between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// The same generator when counter words 1..3 are fixed for the whole walk:
// the first round's product of word 2 is precomputed (pre_x = hi1 ^ c1 ^ k0,
// pre_y = lo1), leaving one product in round one.
__device__ __forceinline__ uint4 philox4x32_10_pre(uint32_t c0, uint32_t c3, uint32_t pre_x,
                                                   uint32_t pre_y, uint32_t k0, uint32_t k1) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    uint4 c = make_uint4(pre_x, pre_y, hi0 ^ c3 ^ k1, lo0);
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
        const uint32_t h0 = __umulhi(0xD2511F53u, c.x), l0 = 0xD2511F53u * c.x;
        const uint32_t h1 = __umulhi(0xCD9E8D57u, c.z), l1 = 0xCD9E8D57u * c.z;
        c = make_uint4(h1 ^ c.y ^ k0, l1, h0 ^ c.w ^ k1, l0);
    }
    return c;
}

// The float 1.m whose mantissa m is the low 23 bits of w:
// (w & 0x007fffff) | 0x3f800000 as one three-input logic operation, the
// exponent bits held in a register (two immediates would take two).
__device__ __forceinline__ float mant_one(uint32_t w) {
    uint32_t r;
    asm("lop3.b32 %0, %1, 0x007fffff, %2, 0xEA;" : "=r"(r) : "r"(w), "r"(0x3f800000u));
    return __uint_as_float(r);
}

// 32 x 32 -> 64-bit product as one wide multiply.
__device__ __forceinline__ void mul_wide(uint32_t a, uint32_t b, uint32_t &lo, uint32_t &hi) {
    uint64_t p;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(b));
    lo = (uint32_t)p;
    hi = (uint32_t)(p >> 32);
}

// Philox4x32-10 with the ten round keys given (rk0[r] = k0 + r 0x9E3779B9,
// rk1[r] = k1 + r 0xBB67AE85); with counter words 1..3 fixed for a walk the
// first round's product of word 2 is precomputed (pre_x = hi ^ c1 ^ rk0[0],
// pre_y = lo of 0xCD9E8D57 * c2).
__device__ __forceinline__ uint4 philox_rk_pre(uint32_t c0, uint32_t c3, uint32_t pre_x,
                                               uint32_t pre_y, const uint32_t (&rk0)[10],
                                               const uint32_t (&rk1)[10]) {
    uint32_t lo0, hi0;
    mul_wide(0xD2511F53u, c0, lo0, hi0);
    uint4 c = make_uint4(pre_x, pre_y, hi0 ^ c3 ^ rk1[0], lo0);
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        uint32_t l0, h0, l1, h1;
        mul_wide(0xD2511F53u, c.x, l0, h0);
        mul_wide(0xCD9E8D57u, c.z, l1, h1);
        c = make_uint4(h1 ^ c.y ^ rk0[r], l1, h0 ^ c.w ^ rk1[r], l0);
    }
    return c;
}

__device__ __forceinline__ uint4 philox_rk(uint4 c, const uint32_t (&rk0)[10],
                                           const uint32_t (&rk1)[10]) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t l0, h0, l1, h1;
        mul_wide(0xD2511F53u, c.x, l0, h0);
        mul_wide(0xCD9E8D57u, c.z, l1, h1);
        c = make_uint4(h1 ^ c.y ^ rk0[r], l1, h0 ^ c.w ^ rk1[r], l0);
    }
    return c;
}

// Shared-memory layout of one CTA: model tables, then for each warp its
// exit-record ring and its scheduler state.  A walker W states what it
// records per material: W::Occ (step counts, or occupation times when they
// can be fractional) for W::kStored materials (all but material 0 when that
// one is derived from the step total, else all K), and W::kHist words per
// lane of shared-memory occupation histogram (W::HistT).
template <class W>
struct Ring {
    using Real = typename W::Real;
    Real x[kRing], z[kRing], th[kRing];
    uint32_t meta[kRing];  // wall | m_last << 2 | truncated << 6 | model << 8
    int32_t item[kRing];
    uint32_t n[kRing];     // occupation steps (all steps but the exiting one)
    uint32_t path[kRing];
    uint32_t aux[kRing];   // interface randomisations (TM walks)
    typename W::Occ cnt[W::kStored][kRing];
};

// Scheduler state of one warp (every field is the same for all its lanes,
// each lane reads back what it wrote), kept out of registers because only
// the exit handler touches it.
struct WarpState {
    unsigned long long steps[32];
    unsigned long long walks, trunc;
    double nx0, nz0;
    int32_t disp_item, disp_rem, disp_model;
    uint32_t disp_next, nid;
    uint32_t head, tail;
    int32_t queue_empty;
    int32_t home;  // grouped launches: the queue this warp takes items from
};

// The model's rates [E][K] and boundary constants [E], staged in shared
// memory ahead of the warps' areas; sized by the model's E and K.
struct SharedTables {
    double *kappa;
    EvalDev *ev;
};

__host__ __device__ constexpr size_t tables_bytes(int E, int K) {
    return ((size_t)E * K * sizeof(double) + 15) / 16 * 16 + (size_t)E * sizeof(EvalDev);
}

template <class W>
struct WarpSmem {
    Ring<W> ring;
    WarpState st;
    typename W::HistT hist[W::kHist][32];     // per-lane occupation histogram
    float4 tail[W::kCoop ? 64 : 1];           // step increments of the cooperative tail
};

// A warp whose queue is drained switches to the cooperative tail once it
// has at most this many walks left.
constexpr int kTailWalks = 8;


template <class W>
__host__ __device__ constexpr size_t shared_bytes(int warps, int E, int K) {
    return (tables_bytes(E, K) + 15) / 16 * 16 + (size_t)warps * sizeof(WarpSmem<W>);
}

// Exit information handed from a walker to the scheduler.
template <class Real>
struct ExitInfo {
    Real x, z, th;  // exit point (walker coordinates) and hit fraction
    int wall;       // 0..3
    int mlast;      // material of the last point inside
    uint32_t nocc;  // occupation steps (all steps but the exiting one)
    uint32_t aux;   // interface randomisations (TM walks)
};

// Scheduler kernel.  W is a walker type providing
//   using Real; static constexpr int KMAX;
//   start(M, A, x0, z0, path, node_id, model)  -- begin a walk
//   iterate(M, A, path, ExitInfo&) -> 0 running, 1 exited, 2 truncated
//     (a few Euler steps per call; max_steps is a multiple of them)
//   counts(M, nocc, c): steps spent in materials 1..KMAX-1 (at the exit,
//     after nocc occupation steps)
//   bind(a): shared-memory address of the lane's occupancy histogram
//   static sample(M, T, A, model, e, x, z, th, wall, mlast, counts) -> double2
//   static to_abs(M, x, z, ax, az)
//   kGrouped: takes items from per-model queues (multi-model launches)
//   kMinCTAs: CTAs of 256 threads that must fit on an SM (the register bound)
// Launch bounds: at most 256 threads, and at least W::kMinCTAs such CTAs per
// SM: 3 leaves up to 85 registers a thread, 4 leaves 64.
template <class W>
__global__ void __launch_bounds__(256, W::kMinCTAs) walk_kernel(const __grid_constant__ ModelDev M,
                                                   const WalkArgs A) {
    using Real = typename W::Real;
    constexpr int KMAX = W::KMAX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SharedTables T;
    T.kappa = reinterpret_cast<double *>(smem_raw);
    T.ev = reinterpret_cast<EvalDev *>(smem_raw + ((size_t)M.E * M.K * sizeof(double) + 15) / 16 * 16);
    WarpSmem<W> &WS = reinterpret_cast<WarpSmem<W> *>(
        smem_raw + (tables_bytes(M.E, M.K) + 15) / 16 * 16)[threadIdx.x >> 5];
    Ring<W> &R = WS.ring;
    WarpState &S = WS.st;

    for (int i = threadIdx.x; i < M.E * M.K; i += blockDim.x) T.kappa[i] = M.kappa[i];
    for (int i = threadIdx.x; i < M.E; i += blockDim.x) T.ev[i] = M.ev[i];

    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const bool dump = A.rec_steps != nullptr;
    S.steps[lane] = 0ull;
    if (lane == 0) {
        S.walks = 0ull; S.trunc = 0ull;
        S.disp_item = -1; S.disp_rem = 0; S.disp_model = 0; S.disp_next = 0; S.nid = 0;
        S.head = S.tail = 0;
        S.queue_empty = 0;
        S.nx0 = S.nz0 = 0.0;
        S.home = 0;
        if (W::kGrouped && A.qbase) {
            const float x = ((float)blockIdx.x + 0.5f) / (float)gridDim.x;
            int m = 0;
            while (m + 1 < A.n_queues && A.home_cut[m + 1] <= x) ++m;
            S.home = m;
        }
    }
    __syncthreads();

    // per-lane walk state
    W w;
    w.bind(&WS.hist[0][lane]);
    bool active = false;
    int item = 0;
    int model = 0;
    uint32_t path = 0;

    // Turn records [head, head + cnt) of the ring into samples; lane l
    // handles evaluation l mod Epad of records l / Epad, l / Epad + 32 / Epad,
    // ...; the samples of each item are summed across the lanes in a fixed
    // shuffle order and lane e adds them to the item's slot for evaluation e.
    auto process = [&](int cnt) {
        const int Epad = M.Epad;
        const int my_e = lane & (Epad - 1);
        const int my_ro = lane / Epad;
        const int per_round = 32 / Epad;
        const uint32_t head = S.head;
        const int rounds = (cnt * Epad + 31) >> 5;
        for (int k = 0; k < rounds; ++k) {
            const int ri = k * per_round + my_ro;
            double2 v = make_double2(0.0, 0.0);
            int my_it = -1;
            if (ri < cnt && my_e < M.E) {
                const int s = (head + ri) & (kRing - 1);
                const uint32_t meta = R.meta[s];
                const bool tr = (meta >> 6) & 1u;
                typename W::Occ c[KMAX];
                if constexpr (W::kStored == KMAX) {
#pragma unroll
                    for (int j = 0; j < KMAX; ++j) c[j] = R.cnt[j][s];
                } else {
                    uint32_t rest = R.n[s];
#pragma unroll
                    for (int j = 1; j < KMAX; ++j) {
                        c[j] = R.cnt[j - 1][s];
                        rest -= c[j];
                    }
                    c[0] = rest;
                }
                if (dump) {
                    if (my_e == 0) {
                        const int64_t o = (int64_t)(R.path[s] - A.items[0].path0);
                        double ex, ez;
                        W::to_abs(M, R.x[s], R.z[s], ex, ez);
                        A.rec_steps[o] = (int64_t)R.n[s] + (tr ? 0 : 1);
#pragma unroll
                        for (int j = 0; j < KMAX; ++j)
                            if (j < M.K) {
                                if (A.rec_counts) A.rec_counts[o * M.K + j] = (int64_t)c[j];
                                if (A.rec_occ) A.rec_occ[o * M.K + j] = (double)c[j];
                            }
                        if (A.rec_hits) A.rec_hits[o] = (int64_t)R.aux[s];
                        A.rec_exit[3 * o + 0] = ex;
                        A.rec_exit[3 * o + 1] = ez;
                        A.rec_exit[3 * o + 2] = (double)R.th[s];
                        A.rec_wall[o] = tr ? -1 : (int)(meta & 3u);
                        A.rec_mlast[o] = (int)((meta >> 2) & 7u);
                    }
                } else if (!tr) {
                    v = W::sample(M, T, A, (int)(meta >> 8), my_e, R.x[s], R.z[s], R.th[s],
                                  (int)(meta & 3u), (int)((meta >> 2) & 7u), c);
                    my_it = R.item[s];
                }
            }
            unsigned pend = __ballot_sync(kFull, my_it >= 0);
            while (pend) {
                const int it = __shfl_sync(kFull, my_it, __ffs(pend) - 1);
                const bool mine = my_it == it;
                double a0 = mine ? v.x : 0.0, a1 = mine ? v.y : 0.0;
                double a2 = a0 * a0, a3 = a1 * a1;
                for (int off = 16; off >= Epad; off >>= 1) {
                    a0 += __shfl_xor_sync(kFull, a0, off);
                    a1 += __shfl_xor_sync(kFull, a1, off);
                    a2 += __shfl_xor_sync(kFull, a2, off);
                    a3 += __shfl_xor_sync(kFull, a3, off);
                }
                if (lane < M.E) {
                    double *o = A.slots + ((size_t)it * M.E + lane) * 4;
                    o[0] += a0;
                    o[1] += a1;
                    o[2] += a2;
                    o[3] += a3;
                }
                pend &= ~__ballot_sync(kFull, mine);
            }
        }
        __syncwarp();
        S.head = head + (uint32_t)cnt;
        __syncwarp();
    };

    // Hand paths to idle lanes, opening the next queued item whenever the
    // current one is fully handed out.
    auto refill = [&]() {
        unsigned need = __ballot_sync(kFull, !active);
        if (A.cancel && need) {
            // a cancelled request: no more paths; the walks in flight end
            int c = 0;
            if (lane == 0) c = *reinterpret_cast<const volatile int32_t *>(A.cancel);
            if (__shfl_sync(kFull, c, 0)) {
                if (lane == 0) {
                    S.queue_empty = 1;
                    S.disp_rem = 0;
                }
                __syncwarp();
                return;
            }
        }
        while (need) {
            if (S.disp_rem == 0) {
                if (S.queue_empty) break;
                int it = -1;
                if (lane == 0) {
                    if (W::kGrouped && A.qbase) {
                        // the home queue first, then the next ones in turn
                        int m = S.home;
                        for (int t = 0; t < A.n_queues; ++t) {
                            const int q = atomicAdd(A.queue + m, 1);
                            if (q < A.qbase[m + 1] - A.qbase[m]) {
                                it = A.order[A.qbase[m] + q];
                                break;
                            }
                            m = m + 1 == A.n_queues ? 0 : m + 1;
                        }
                        S.home = m;
                    } else {
                        const int q = atomicAdd(A.queue, 1);
                        if (q < A.n_items) it = A.order ? A.order[q] : q;
                    }
                }
                it = __shfl_sync(kFull, it, 0);
                if (it < 0) {
                    if (lane == 0) S.queue_empty = 1;
                    __syncwarp();
                    break;
                }
                const Item I = A.items[it];
                if (!dump) {
                    if (lane < M.E) {
                        double *o = A.slots + ((size_t)it * M.E + lane) * 4;
                        o[0] = 0.0; o[1] = 0.0; o[2] = 0.0; o[3] = 0.0;
                    }
                    if (lane == 0) A.item_trunc[it] = 0;
                }
                if (lane == 0) {
                    S.disp_item = it;
                    S.disp_model = I.model;
                    S.disp_next = I.path0;
                    S.disp_rem = I.count;
                    S.nx0 = A.nodes[2 * I.node];
                    S.nz0 = A.nodes[2 * I.node + 1];
                    S.nid = A.node_ids ? A.node_ids[I.node] : (uint32_t)I.node;
                }
                __syncwarp();
                if (I.count == 0) continue;
            }
            const int rem = S.disp_rem;
            const int navail = __popc(need);
            const int k = navail < rem ? navail : rem;
            const int rank = __popc(need & lt_mask);
            const bool mine = ((need >> lane) & 1u) && rank < k;
            if (mine) {
                path = S.disp_next + (uint32_t)rank;
                item = S.disp_item;
                model = S.disp_model;
                active = true;
                w.start(M, A, S.nx0, S.nz0, path, S.nid, model);
            }
            const unsigned got = __ballot_sync(kFull, mine);
            need &= ~got;
            if (lane == 0) {
                S.disp_next += (uint32_t)k;
                S.disp_rem = rem - k;
            }
            __syncwarp();
        }
    };

    // Records of the walks that ended this iteration (st: 1 exited,
    // 2 truncated), then a batch of samples once 32 records are waiting.
    ExitInfo<Real> ei{};
    auto on_exits = [&](int st) {
        const unsigned em = __ballot_sync(kFull, st != 0);
        const int nex = __popc(em);
        if (st != 0) active = false;
        const uint32_t tail = S.tail;
        if (st != 0) {
            const int slot = (tail + __popc(em & lt_mask)) & (kRing - 1);
            const bool tr = st == 2;
            R.x[slot] = ei.x;
            R.z[slot] = ei.z;
            R.th[slot] = ei.th;
            R.meta[slot] = (uint32_t)ei.wall | ((uint32_t)ei.mlast << 2) | ((uint32_t)tr << 6) |
                           ((uint32_t)model << 8);
            R.item[slot] = item;
            R.n[slot] = ei.nocc;
            R.path[slot] = path;
            R.aux[slot] = ei.aux;
            typename W::Occ c[W::kStored];
            w.counts(M, ei.nocc, c);
#pragma unroll
            for (int j = 0; j < W::kStored; ++j) R.cnt[j][slot] = c[j];
            S.steps[lane] += (unsigned long long)ei.nocc + (tr ? 0ull : 1ull);
            if (tr && !dump) atomicAdd(&A.item_trunc[item], 1);
        }
        const unsigned trm = __ballot_sync(kFull, st == 2);
        if (lane == 0) {
            S.tail = tail + (uint32_t)nex;
            S.walks += (unsigned long long)nex;
            S.trunc += (unsigned long long)__popc(trm);
        }
        __syncwarp();
        while (S.tail - S.head >= 32) process(32);
    };

    refill();
    int n_active = __popc(__ballot_sync(kFull, active));
    while (n_active > 0) {
        if (W::kCoop && n_active <= kTailWalks && S.queue_empty && S.disp_rem == 0) break;
        int st = 0;
        if (active) st = w.iterate(M, A, path, ei);
        if (__ballot_sync(kFull, st != 0) == 0) continue;
        on_exits(st);
        refill();
        n_active = __popc(__ballot_sync(kFull, active));
    }

    // Cooperative tail: nothing is left to hand out and at most kTailWalks
    // walks remain.  Each round, lane l computes Philox pair l / a of the
    // (l mod a)-th live walk (a walks live), so every walk gets 32 / a pairs
    // of step increments at once; then each live lane runs its 2 (32 / a)
    // steps from shared memory, whose serial part is only the move, the wall
    // tests and the material lookup.
    if constexpr (W::kCoop) {
        float4 *buf = WS.tail;
        while (n_active > 0) {
            const unsigned act = __ballot_sync(kFull, active);
            const int a = __popc(act);
            const int per = 32 / a;
            const int j = lane % a, q = lane / a;
            unsigned m = act;
            for (int t = 0; t < j; ++t) m &= m - 1u;
            const int src = __ffs(m) - 1;
            const uint32_t n0 = __shfl_sync(kFull, w.steps(), src);
            const uint2 k0 = w.key();
            const uint2 key = make_uint2(__shfl_sync(kFull, k0.x, src), __shfl_sync(kFull, k0.y, src));
            if (q < per) W::pair_increments(A, n0, key, (uint32_t)q, buf[j * 2 * per + 2 * q],
                                            buf[j * 2 * per + 2 * q + 1]);
            __syncwarp();
            int st = 0;
            if (active) st = w.consume(M, A, buf + __popc(act & lt_mask) * 2 * per, 2 * per, ei);
            __syncwarp();
            if (__ballot_sync(kFull, st != 0) != 0) on_exits(st);
            n_active = __popc(__ballot_sync(kFull, active));
        }
    }
    if (S.tail != S.head) process((int)(S.tail - S.head));
    // every item handed to this warp has been flushed (its walks all ended)

    unsigned long long my_steps = S.steps[lane];
    for (int off = 16; off > 0; off >>= 1) my_steps += __shfl_xor_sync(kFull, my_steps, off);
    if (lane == 0 && !dump) {
        atomicAdd(&A.counters[0], my_steps);
        atomicAdd(&A.counters[1], S.walks);
        atomicAdd(&A.counters[2], S.trunc);
    }
}

}  // namespace sdd
