// rn_kernels.cuh -- kernel templates of the annealing path (instantiated in
// rn_anneal{1,2,4}.cu, rn_batch.cu and rn_kernels.cu).
//
//   evaluate_kernel        Simulate(x) of Table 1 for a batch of vectors, warp each
//   evaluate_smem_kernel   the same with the shared-memory tables (N > 128)
//   anneal_kernel          persistent annealing kernel, warp per chain (Table 1
//                          inner loop: GetCandidate, Simulate, Metropolis
//                          acceptance), register tables
//   anneal_smem_kernel     the same with shared-memory tables
//   anneal_batch_kernel    one persistent launch over every chain of many networks
//
// Shared memory of a block: a code region (1 KiB per warp: the 16-bit state
// codes of the warp's nodes, so that every code offset fits the table words),
// then one region per warp (x, constraint counters, and for the shared-memory
// path the table words and per-node update state).
#pragma once

#include "rn_device.cuh"
#include "rn_launch.h"
#include "rn_smem.cuh"

namespace rn {

__host__ __device__ inline uint32_t round16(uint32_t v) { return (v + 15u) & ~15u; }

// Region of one warp after the code region.
struct WarpRegion {
    uint32_t lut_words;   // shared-memory path: table words (0 for the register path)
    uint32_t bytes;       // total bytes (multiple of 16)
};

__host__ __device__ inline WarpRegion warp_region(bool smem_path, const int *D, int npl,
                                                  int pstride, int N)
{
    WarpRegion r;
    if (smem_path) {
        r.lut_words = smem_path_lut_words(D, npl);
        r.bytes = round16(smem_path_warp_bytes(r.lut_words, npl, pstride, N));
    } else {
        r.lut_words = 0;
        r.bytes = round16((uint32_t)pstride + 2u * round16((uint32_t)N));
    }
    return r;
}

// ------------------------------------------------------ register table path --
template <int NPL, int CG, int D0, int D1>
struct RegPath {
    Regs<NPL, D0, D1> R;
    uint8_t *sm;
    uint32_t codes;       // offset of the warp's code array (256-byte aligned)
    // undo record of the owner lane
    int undo_kd, undo_kind, undo_slot;
    uint32_t undo_val;

    __device__ void load(const DevNet &net, const int8_t *x, int lane)
    {
        load_regs<NPL, D0, D1>(R, net, x, lane);
    }

    __device__ void change_edge(const DevNet &, int lane, int owner, int pos, int w, int p, int t,
                                int)
    {
        if (lane != owner) return;
        const int kd = ((pos >> 8) & 0xff) * 32 + (pos & 0xff);
        uint32_t old = 0;
        for_each_word<NPL, D0, D1>(R, [&](int k, int d, uint32_t &word) {
            old = (k * 32 + d == kd) ? word : old;
        });
        undo_kd = kd;
        undo_kind = 0;
        undo_val = old;
        const uint32_t nw = edge_word(w, p, t, old >> 24);
        for_each_word<NPL, D0, D1>(R, [&](int k, int d, uint32_t &word) {
            word = (k * 32 + d == kd) ? nw : word;
        });
    }

    __device__ void change_node(int lane, int owner, int slot, int kind, int v)
    {
        if (lane != owner) return;
        undo_kind = kind;
        undo_slot = slot;
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
            if (k != slot) continue;
            if (kind == 3) { undo_val = (uint32_t)R.u[k]; R.u[k] = v; }
            else if (kind == 4) { undo_val = (uint32_t)R.m1[k]; R.m1[k] = v + 1; }
            else { undo_val = (uint32_t)R.d2[k]; R.d2[k] = v == 2; }
        }
    }

    __device__ void undo(int lane, int owner)
    {
        if (lane != owner) return;
        if (undo_kind == 0) {
            const int kd = undo_kd;
            const uint32_t ov = undo_val;
            for_each_word<NPL, D0, D1>(R, [&](int k, int d, uint32_t &word) {
                word = (k * 32 + d == kd) ? ov : word;
            });
            return;
        }
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
            if (k != undo_slot) continue;
            if (undo_kind == 3) R.u[k] = (int32_t)undo_val;
            else if (undo_kind == 4) R.m1[k] = (int32_t)undo_val;
            else R.d2[k] = (int32_t)undo_val;
        }
    }

    __device__ int32_t simulate(const DevNet &net, int lane, uint8_t *traj,
                                int32_t limit = INT32_MAX)
    {
        return rn::simulate<NPL, CG, D0, D1>(R, net, sm, codes, lane, traj, limit);
    }
};

// ---------------------------------------------------------------- evaluate --
template <int NPL, int CG, int D0, int D1>
__global__ void __launch_bounds__(128) evaluate_kernel(DevNet net, const int8_t *__restrict__ X,
                                                       int64_t xstride, int32_t n,
                                                       int32_t *__restrict__ score,
                                                       int32_t *__restrict__ score2,
                                                       uint8_t *__restrict__ traj)
{
    extern __shared__ __align__(256) uint8_t sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    RegPath<NPL, CG, D0, D1> P;
    P.sm = sm;
    P.codes = (uint32_t)warp * kCodeBytesPerWarp;
    for (int v = blockIdx.x * wpb + warp; v < n; v += gridDim.x * wpb) {
        P.load(net, X + (size_t)v * xstride, lane);
        uint8_t *tv = traj ? traj + (size_t)v * net.C * net.T * net.N : nullptr;
        const int32_t y = P.simulate(net, lane, tv);
        if (lane == 0) {
            score[v] = y;
            if (score2) score2[v] = y;
        }
        __syncwarp();
    }
}

__device__ __forceinline__ SmemPath make_smem_path(const DevNet &net, uint8_t *sm, int warp,
                                                   int wpb, uint32_t region_bytes,
                                                   uint32_t lut_words)
{
    SmemPath P;
    P.sm = sm;
    P.codes = (uint32_t)warp * kCodeBytesPerWarp;
    uint8_t *region = sm + (uint32_t)wpb * kCodeBytesPerWarp + (uint32_t)warp * region_bytes;
    P.lut = reinterpret_cast<uint32_t *>(region);
    P.node = P.lut + lut_words;
    P.npl = net.npl;
    return P;
}

// -------------------------------------------------------------- annealing --

// Domain of parameter kind k (Section 2.1: w, p, t; Section 2.2: u, m, d).
__device__ __forceinline__ int domain(int kind, bool fast, int8_t (&vals)[6])
{
    switch (kind) {
    case 0: vals[0] = 0; vals[1] = 1; vals[2] = 2; return 3;
    case 1: vals[0] = -1; vals[1] = 0; vals[2] = 1; return 3;
    case 2: vals[0] = 1; vals[1] = 2; return 2;
    case 3:
        if (fast) { vals[0] = 10; vals[1] = 11; vals[2] = 12; return 3; }
#pragma unroll
        for (int k = 0; k < 6; ++k) vals[k] = (int8_t)(k + 1);
        return 6;
    case 4: vals[0] = 0; vals[1] = 1; vals[2] = 2; return 3;
    default: vals[0] = 1; vals[1] = 2; return 2;
    }
}

// Rebuild the per-chain constraint counters of Section 2.5.3 from x.
__device__ __forceinline__ void count_constraints(const DevNet &net, const int8_t *x,
                                                  uint8_t *out_nz, uint8_t *pos_in, int lane)
{
    for (int i = lane; i < net.N; i += 32) {
        int o = 0, q = 0;
        for (int k = net.out_ptr[i]; k < net.out_ptr[i + 1]; ++k) o += x[net.out_edges[k]] != 0;
        for (int k = net.in_ptr[i]; k < net.in_ptr[i + 1]; ++k) {
            const int e = net.in_edges[k];
            q += (x[e] != 0) && (x[net.E + e] == 1);
        }
        out_nz[i] = (uint8_t)min(o, 255);
        pos_in[i] = (uint8_t)min(q, 255);
    }
}

// GetCandidate (Table 1) for a network with free parameters: the pick(r0)-th
// free parameter j, then the pick(r1)-th of its domain values != x_j whose
// single change keeps both constraints of Section 2.5.3 (counters out_nz,
// pos_in of x).  Returns false for a null move (no such value).  `xr(j)`
// reads x_j (shared memory, or global memory through L2).  With LANES_DIFFER
// (lanes of one warp draw different candidates, so their parameter kinds
// differ) the constraint inputs are read for every kind and combined without
// branches; otherwise (one candidate per warp) only the kinds that need them
// read them, and the value is found by walking the listed domain.
template <bool LANES_DIFFER = false, class XR>
__device__ __forceinline__ bool get_candidate_x(const DevNet &net, XR xr, const uint8_t *out_nz,
                                                const uint8_t *pos_in, uint32_t r0, uint32_t r1,
                                                int &j, int &kind, int &idx, int &cur, int &v)
{
    const int E = net.E, N = net.N;
    j = net.free_list[pick(r0, (uint32_t)net.n_free)];
    param_kind(j, E, N, kind, idx);
    cur = xr(j);
    if constexpr (LANES_DIFFER) {
        // an edge parameter's own edge, edge 0 for a node parameter (read and
        // unused: a loaded network has at least one edge)
        const int ie = kind < 3 ? idx : 0;
        const int a = net.src[ie], b = net.dst[ie];
        const bool out_low = out_nz[a] < 2, pos_low = pos_in[b] < 2;
        const bool p_pos = xr(E + ie) == 1, w_nz = xr(ie) != 0;
        const bool blocked0 = (kind == 0) & (cur != 0) & (out_low | (p_pos & pos_low));
        const bool blocked_all = (kind == 1) & (cur == 1) & w_nz & pos_low;
        const bool fast = (kind == 3) & (net.fast[kind == 3 ? idx : 0] != 0);
        return pick_alternative(kind, fast, cur, blocked0, blocked_all, r1, v);
    } else {
        // the domain's listed values, walked (measured a little faster than the
        // arithmetic choice where the whole warp holds one candidate)
        int8_t vals[6];
        const int nd = domain(kind, kind == 3 && net.fast[idx], vals);
        bool blocked0 = false, blocked_all = false;
        if (kind == 0 && cur != 0) {
            const int a = net.src[idx], b = net.dst[idx];
            blocked0 = out_nz[a] < 2 || (xr(E + idx) == 1 && pos_in[b] < 2);
        } else if (kind == 1 && cur == 1 && xr(idx) != 0) {
            blocked_all = pos_in[net.dst[idx]] < 2;
        }
        int8_t alts[6];
        int n_alt = 0;
        if (!blocked_all) {
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                if (k >= nd) break;
                const int a = vals[k];
                if (a == cur || (blocked0 && a == 0)) continue;
                alts[n_alt++] = (int8_t)a;
            }
        }
        if (n_alt == 0) return false;
        v = alts[pick(r1, (uint32_t)n_alt)];
        return true;
    }
}

template <bool LANES_DIFFER = false>
__device__ __forceinline__ bool get_candidate(const DevNet &net, const int8_t *xs,
                                              const uint8_t *out_nz, const uint8_t *pos_in,
                                              uint32_t r0, uint32_t r1, int &j, int &kind,
                                              int &idx, int &cur, int &v)
{
    return get_candidate_x<LANES_DIFFER>(net, [&](int k) { return (int)xs[k]; }, out_nz, pos_in,
                                         r0, r1, j, kind, idx, cur, v);
}

// Constraint counters after x_j: cur -> v (x still holds cur); xr as above.
template <class XR>
__device__ __forceinline__ void apply_counters_x(const DevNet &net, XR xr, uint8_t *out_nz,
                                                 uint8_t *pos_in, int kind, int idx, int cur,
                                                 int v)
{
    const int E = net.E;
    if (kind == 0 && (cur == 0) != (v == 0)) {
        const int delta = v != 0 ? 1 : -1;
        out_nz[net.src[idx]] += delta;
        if (xr(E + idx) == 1) pos_in[net.dst[idx]] += delta;
    } else if (kind == 1 && xr(idx) != 0) {
        if (cur == 1) pos_in[net.dst[idx]] -= 1;
        if (v == 1) pos_in[net.dst[idx]] += 1;
    }
}

__device__ __forceinline__ void apply_counters(const DevNet &net, const int8_t *xs,
                                               uint8_t *out_nz, uint8_t *pos_in, int kind,
                                               int idx, int cur, int v)
{
    apply_counters_x(net, [&](int k) { return (int)xs[k]; }, out_nz, pos_in, kind, idx, cur, v);
}

// Largest dE the acceptance word r accepts at level l (Table 1: r < thr(T_l,
// dE)); the thresholds do not increase with dE, so the accepted dE >= 1 form
// a prefix of the level's table.  0 if r accepts no uphill move.
__device__ __forceinline__ int32_t max_accepted_dE(const DevSched &sc, int64_t l, uint32_t r)
{
    const uint32_t *t = sc.thr + sc.thr_off[l];   // t[dE - 1]
    int lo = 0, hi = sc.thr_len[l];
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (r < __ldg(t + mid - 1)) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void warp_copy16(void *dst, const void *src, int bytes, int lane)
{
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    for (int k = lane; k < (bytes >> 4); k += 32) d[k] = s[k];
}

// Chain state moves between warps of different SMs from one work item to the
// next: read it from L2 (never from a possibly stale L1 line) ...
__device__ __forceinline__ void warp_load_cg(void *dst, const void *src, int bytes, int lane)
{
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    for (int k = lane; k < (bytes >> 4); k += 32) d[k] = __ldcg(s + k);
}

// ... and write it to L2.
__device__ __forceinline__ void warp_store_cg(void *dst, const void *src, int bytes, int lane)
{
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    for (int k = lane; k < (bytes >> 4); k += 32) __stcg(d + k, s[k]);
}

// Wait (bounded: LIMIT polls) until `done` reaches `need`; false if the wait
// gave up or another warp reported a failure.  One lane polls; the result is
// broadcast.
template <int LIMIT = kWaitLimit>
__device__ __forceinline__ bool wait_for_chunk(const int32_t *done, int need, int32_t *err,
                                               int lane)
{
    int ok = 1;
    if (lane == 0) {
        const volatile int32_t *flag = done;
        const volatile int32_t *failed = err;
        int polls = 0;
        while (*flag < need) {
            if (*failed) {
                ok = 0;
                break;
            }
            if (++polls > LIMIT) {
                ok = 0;
                atomicExch(err, 1);
                break;
            }
            __nanosleep(256);
        }
        __threadfence();
    }
    return __shfl_sync(kFull, ok, 0) != 0;
}

// Steps [g_lo, g_hi) of one chain (Table 1 inner loop), its state in and out
// of global memory through L2, then the chain's chunk counter is published.
// EARLY_OK compiles exact early rejection in; the batched kernel leaves it out
// (one simulation instance per table path keeps that kernel's code small).
template <typename Path, bool EARLY_OK = true>
__device__ __forceinline__ void run_chunk(Path &P, const DevNet &net, const DevChains &ch,
                                          const DevSched &sc, int chain, int64_t g_lo,
                                          int64_t g_hi, int8_t *xs, uint8_t *out_nz,
                                          uint8_t *pos_in, int32_t *done_flag, int done_value,
                                          int lane)
{
    const int E = net.E;
    int8_t *xg = ch.x_cur + (size_t)chain * ch.pstride;
    int8_t *xb = ch.x_best + (size_t)chain * ch.pstride;
    warp_load_cg(xs, xg, ch.pstride, lane);
    __syncwarp();
    P.load(net, xs, lane);
    count_constraints(net, xs, out_nz, pos_in, lane);
    __syncwarp();
    int32_t d_cur = __ldcg(ch.d_cur + chain), d_best = __ldcg(ch.d_best + chain);
    int32_t n_acc = 0, n_up = 0, n_null = 0;

    int64_t level = g_lo / sc.iters;
    int64_t in_level = g_lo - level * sc.iters;
    for (int64_t g = g_lo; g < g_hi; ++g) {
        if (in_level == sc.iters) {
            in_level = 0;
            ++level;
        }
        if (sc.reset_to_best && in_level == 0) {
            // Table 1: every level starts from the chain's x_best
            warp_load_cg(xs, xb, ch.pstride, lane);
            __syncwarp();
            P.load(net, xs, lane);
            count_constraints(net, xs, out_nz, pos_in, lane);
            __syncwarp();
            d_cur = d_best;
        }
        ++in_level;
        const uint4 r = philox(ch.seed, (uint32_t)g, (uint32_t)((uint64_t)g >> 32),
                               (uint32_t)chain, 0u);
        if (net.n_free == 0) {
            ++n_null;
            continue;
        }
        int j, kind, idx, cur, v;
        if (!get_candidate(net, xs, out_nz, pos_in, r.x, r.y, j, kind, idx, cur, v)) {
            ++n_null;
            continue;
        }

        // apply the candidate to the owner lane's table entry
        int owner;
        if (kind < 3) {
            const int pos = net.edge_pos[idx];
            owner = pos >> 16;
            int w = xs[idx], p = xs[E + idx], t = xs[2 * E + idx];
            if (kind == 0) w = v; else if (kind == 1) p = v; else t = v;
            P.change_edge(net, lane, owner, pos, w, p, t, idx);
        } else {
            const int q = net.node_q[idx];
            owner = q / net.npl;
            P.change_node(lane, owner, q - owner * net.npl, kind, v);
        }
        __syncwarp();
        const int64_t l = level - sc.level0;
        // with exact early rejection the simulation may stop once the candidate
        // cannot be accepted: above d_cur + the largest dE this draw accepts
        const int32_t limit =
            EARLY_OK && sc.early_reject ? d_cur + max_accepted_dE(sc, l, r.z) : INT32_MAX;
        const int32_t d_cand = P.simulate(net, lane, nullptr, limit);

        // Metropolis acceptance against the host-computed threshold table
        const int32_t dE = d_cand - d_cur;
        bool accept = dE <= 0;
        if (!accept) {
            if (dE <= sc.thr_len[l]) accept = r.z < __ldg(sc.thr + sc.thr_off[l] + dE - 1);
        }
        if (accept) {
            if (lane == 0) {
                apply_counters(net, xs, out_nz, pos_in, kind, idx, cur, v);
                xs[j] = (int8_t)v;
            }
            __syncwarp();
            d_cur = d_cand;
            ++n_acc;
            n_up += dE > 0;
            if (d_cand < d_best) {
                d_best = d_cand;
                warp_store_cg(xb, xs, ch.pstride, lane);
            }
        } else {
            P.undo(lane, owner);
        }
        __syncwarp();
    }
    warp_store_cg(xg, xs, ch.pstride, lane);
    if (lane == 0) {
        __stcg(ch.d_cur + chain, d_cur);
        __stcg(ch.d_best + chain, d_best);
        int64_t *cnt = ch.cnt + 3 * (size_t)chain;
        __stcg(cnt + 0, __ldcg(cnt + 0) + n_acc);
        __stcg(cnt + 1, __ldcg(cnt + 1) + n_up);
        __stcg(cnt + 2, __ldcg(cnt + 2) + n_null);
    }
    // publish: every lane's stores, then the chunk counter of the chain
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicExch(done_flag, done_value);
    __syncwarp();
}

// Three 4-warp blocks per SM (at most 168 registers a thread) unless the
// register tables alone need more room.
template <int NPL, int D0, int D1>
constexpr int anneal_min_blocks()
{
    return D0 + (NPL - 1) * D1 <= 40 ? 3 : 2;
}

// Work item i of a single-network launch: chunk i / n of chain i % n.
template <typename MakePath>
__device__ __forceinline__ void anneal_items(const DevNet &net, const DevChains &ch,
                                             const DevSched &sc, uint8_t *sm,
                                             uint32_t region_bytes, MakePath make_path)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    uint8_t *region = sm + (uint32_t)wpb * kCodeBytesPerWarp + (uint32_t)warp * region_bytes;
    auto P = make_path(warp, wpb);
    const uint32_t lut_bytes = (uint32_t)((uint8_t *)P.node_end() - region);
    int8_t *xs = reinterpret_cast<int8_t *>(region + lut_bytes);
    uint8_t *out_nz = region + lut_bytes + ch.pstride;
    uint8_t *pos_in = out_nz + round16((uint32_t)net.N);
    const int64_t n_items = (int64_t)sc.n_chunks * ch.n;
    for (;;) {
        unsigned int item = 0;
        if (lane == 0) item = atomicAdd(sc.queue, 1u);
        item = __shfl_sync(kFull, item, 0);
        if ((int64_t)item >= n_items) break;
        const int cj = (int)(item / (unsigned)ch.n);
        const int chain = (int)(item - (unsigned)cj * (unsigned)ch.n);
        // chunk cj - 1 of this chain was handed out n items earlier, to a running warp
        if (cj > 0 && !wait_for_chunk(sc.done + chain, cj, sc.err, lane)) return;
        const int64_t g_lo = sc.g0 + (int64_t)cj * sc.chunk;
        const int64_t g_hi = min(sc.g1, g_lo + sc.chunk);
        run_chunk(P, net, ch, sc, chain, g_lo, g_hi, xs, out_nz, pos_in, sc.done + chain, cj + 1,
                  lane);
    }
}

// Register-path wrapper exposing where its (empty) table region ends.
template <int NPL, int CG, int D0, int D1>
struct RegPathR : RegPath<NPL, CG, D0, D1> {
    uint8_t *region;
    __device__ uint8_t *node_end() const { return region; }
};

struct SmemPathR : SmemPath {
    __device__ uint8_t *node_end() const
    {
        return reinterpret_cast<uint8_t *>(node + npl * kF_N * 32);
    }
};

template <int NPL, int CG, int D0, int D1>
__global__ void __launch_bounds__(128, (anneal_min_blocks<NPL, D0, D1>()))
    anneal_kernel(DevNet net, DevChains ch, DevSched sc, uint32_t region_bytes)
{
    extern __shared__ __align__(256) uint8_t sm[];
    anneal_items(net, ch, sc, sm, region_bytes, [&](int warp, int wpb) {
        RegPathR<NPL, CG, D0, D1> P;
        P.sm = sm;
        P.codes = (uint32_t)warp * kCodeBytesPerWarp;
        P.region = sm + (uint32_t)wpb * kCodeBytesPerWarp + (uint32_t)warp * region_bytes;
        return P;
    });
}

template <int NPL, int CG, int D0, int D1>
cudaError_t launch_anneal_t(const DevNet &net, const DevChains &ch, const DevSched &sc,
                            int sm_count, cudaStream_t st)
{
    int wpb = 4;
    const WarpRegion R = warp_region(false, net.D, net.npl, ch.pstride, net.N);
    size_t smem = (size_t)wpb * (kCodeBytesPerWarp + R.bytes);
    auto kern = anneal_kernel<NPL, CG, D0, D1>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wpb * 32, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = sm_count * per_sm;
    if (ch.n > 0 && ch.n < grid * wpb) {
        // fewer chains than resident warps: a block of one warp per chain, which
        // the hardware spreads evenly over the SMs
        wpb = 1;
        grid = ch.n;
        smem = kCodeBytesPerWarp + R.bytes;
    }
    DevSched s = sc;
    plan_chunks(s, ch.n, (int64_t)grid * wpb);
    err = cudaMemsetAsync(s.queue, 0, sizeof(unsigned int), st);
    if (err == cudaSuccess) err = cudaMemsetAsync(s.done, 0, sizeof(int32_t) * (size_t)ch.n, st);
    if (err != cudaSuccess) return err;
    kern<<<grid, wpb * 32, smem, st>>>(net, ch, s, R.bytes);
    return cudaGetLastError();
}

// Register capacities (D0 for slot 0, D1 for the other slots) compiled for the
// annealing kernel; the evaluate kernel uses (16, 16) throughout.
#define RN_ANNEAL_PAIRS(X, NPL_, CG_)                                           \
    X(NPL_, CG_, 4, 4) X(NPL_, CG_, 8, 4) X(NPL_, CG_, 8, 8) X(NPL_, CG_, 12, 8) \
    X(NPL_, CG_, 16, 8) X(NPL_, CG_, 16, 16)

cudaError_t launch_anneal_npl1(const DevNet &net, int d0, int d1, const DevChains &ch,
                               const DevSched &sc, int sm_count, cudaStream_t st);
cudaError_t launch_anneal_npl2(const DevNet &net, int d0, int d1, const DevChains &ch,
                               const DevSched &sc, int sm_count, cudaStream_t st);
cudaError_t launch_anneal_npl4(const DevNet &net, int d0, int d1, const DevChains &ch,
                               const DevSched &sc, int sm_count, cudaStream_t st);

}  // namespace rn
