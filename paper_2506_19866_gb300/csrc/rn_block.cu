// rn_block.cu -- block-per-chain simulation for networks of 513 .. 4096 nodes
// (and smaller ones whose in-degree exceeds the warp paths' 16).
//
// A warp no longer holds the chain: its nodes are spread over the 256 threads
// of a block (node rank r -> slot r / 256, thread r % 256, internal index
// q = thread * npl + slot, 2 <= npl <= 16).  Everything else is the shared-memory
// table path of rn_smem.cuh: table words and per-node byte-SIMD update state
// in shared memory, laid out [..][256] so that each warp's accesses are
// consecutive words, four conditions per group (Sections 2.1-2.3).  The
// priority maximum of a time step is a block maximum (warp redux, then eight
// warp values through shared memory), so each update step has two block
// barriers.  The annealing loop (Table 1: GetCandidate, Simulate, Metropolis)
// runs with thread 0 drawing and deciding and the owner thread of the changed
// table entry applying or undoing it.  The chain's x stays in global memory,
// read through L2 (another SM may have advanced the chain in the previous
// chunk), so that the tables of a 2000-node network fit the block's shared
// memory.  Work items (chunk, chain) come from the same queue scheme as the
// warp kernels, with bounded waits.
#include "rn_kernels.cuh"
#include "rn_screen.h"

namespace rn {
namespace {

constexpr int kBT = 256;        // threads per chain
constexpr int kBW = kBT / 32;   // warps per chain

__device__ __forceinline__ int xcg(const int8_t *x, int j) { return (int)__ldcg(x + j); }

// Shared memory: codes [kBT * npl] u16 at offset 0 (on the register variant,
// which keeps node state in registers for 2, 4, 6 or 8 nodes per thread, a
// second copy of them follows: code_word2), then the table rows, the per-node
// fields (not on the register variant), the constraint counters, a small
// scratch area and, where it fits, the chain's x (xbytes, 0 for none).
struct BlockLayout {
    uint32_t codes, codes2, lut, node, cnt, scratch, x, bytes;
};

__host__ __device__ inline uint32_t round256(uint32_t v) { return (v + 255u) & ~255u; }

__host__ __device__ inline BlockLayout block_layout(const int *D, int npl, int N,
                                                    uint32_t xbytes = 0)
{
    BlockLayout L;
    uint32_t rows = 0;
    for (int k = 0; k < npl; ++k) rows += (uint32_t)groups4(D[k]);
    const uint32_t cb = block_code_bytes(npl);
    const uint32_t node = block_reg_npl(npl) ? 0u : (uint32_t)npl * kF_N * kBT * 4u;
    const uint32_t cnt = round256(2u * (((uint32_t)N + 15u) & ~15u));
    // everything but the codes and x
    const uint32_t rest = rows * kBT * 4u + node + cnt + 256u;
    const bool two = block_reg_npl(npl) && 2u * cb + rest <= kBlockSmemMax;
    L.codes = 0;
    L.codes2 = two ? cb : 0u;
    L.lut = two ? 2u * cb : cb;
    L.node = L.lut + rows * kBT * 4u;
    L.cnt = L.node + node;
    L.scratch = L.cnt + cnt;
    L.x = L.scratch + 256u;
    L.bytes = L.x + xbytes;
    return L;
}

// Broadcast area of the annealing loop (in the scratch region).
struct Bcast {
    uint32_t wmax[kBW][4];   // per-warp maxima of the four conditions' priorities
    uint32_t wsum[kBW];      // per-warp score sums
    uint32_t item;           // work item
    uint32_t rz;             // acceptance word of the step
    int32_t ok;              // a candidate exists (or: the wait succeeded)
    int32_t j, kind, idx, cur, v;   // the candidate x_j: cur -> v (kind, index in its block)
    int32_t owner, pos, w, p, t, slot;   // owner thread and the changed table entry
    int32_t sel[kMaxTop];    // a screened step's moves to simulate
};
static_assert(sizeof(Bcast) <= 256, "the broadcast area is 256 bytes of the layout");

// Constraint counters of Section 2.5.3 from x (global through L2 when `cg`,
// else shared memory).
__device__ void block_count(const DevNet &net, const int8_t *x, int t, uint8_t *out_nz,
                            uint8_t *pos_in, bool cg)
{
    auto X = [&](int j) { return cg ? xcg(x, j) : (int)x[j]; };
    for (int i = t; i < net.N; i += kBT) {
        int o = 0, q = 0;
        for (int k = net.out_ptr[i]; k < net.out_ptr[i + 1]; ++k)
            o += X(net.out_edges[k]) != 0;
        for (int k = net.in_ptr[i]; k < net.in_ptr[i + 1]; ++k) {
            const int e = net.in_edges[k];
            q += (X(e) != 0) && (X(net.E + e) == 1);
        }
        out_nz[i] = (uint8_t)min(o, 255);
        pos_in[i] = (uint8_t)min(q, 255);
    }
}

struct BlockPath {
    uint8_t *sm;
    uint16_t *code;
    uint32_t *lut, *node;
    uint8_t *out_nz, *pos_in;
    Bcast *bc;
    int8_t *xs;   // the chain's x in shared memory (when the launch reserved it)
    int npl;
    uint32_t undo_addr, undo_val;
    bool undo_lut;

    __device__ __forceinline__ uint32_t &F(int k, int f, int t) const
    {
        return node[(k * kF_N + f) * kBT + t];
    }

    __device__ __forceinline__ int lut_row(const DevNet &net, int k, int d) const
    {
        int o = 0;
        for (int kk = 0; kk < k; ++kk) o += groups4(net.D[kk]);
        return o + d;
    }

    // Tables of x (read through L2 when `cg`).
    __device__ void load(const DevNet &net, const int8_t *x, int t, bool cg)
    {
        auto X = [&](int j) { return cg ? xcg(x, j) : (int)x[j]; };
        const int E = net.E, N = net.N;
        int o = 0;
        for (int k = 0; k < npl; ++k) {
            for (int d = 0; d < net.D[k]; ++d) {
                const int e = net.edge_id[(k * net.dtab + d) * kBT + t];
                uint32_t w;
                if (e >= 0)
                    w = edge_word_s(X(e), X(E + e), X(2 * E + e),
                                    2u * (uint32_t)net.node_q[net.src[e]]);
                else
                    w = 0x04040000u | ((uint32_t)(-1 - e) & 0xffffu);
                lut[(o + d) * kBT + t] = w;
            }
            // neutral rows up to a whole group of 4: the code of node 2 t (one
            // bank per lane; npl >= 2 on this path, so node 2 t exists)
            for (int d = net.D[k]; d < groups4(net.D[k]); ++d)
                lut[(o + d) * kBT + t] = 0x04040000u | (4u * (uint32_t)t);
            o += groups4(net.D[k]);
            const int i = net.q_node[t * npl + k];
            uint32_t u = 1, m1 = 1, d2 = 0;
            if (i >= 0) {
                u = net.sync ? 0u : (uint32_t)X(3 * E + i);
                m1 = (uint32_t)X(3 * E + N + i) + 1u;
                d2 = X(3 * E + 2 * N + i) == 2 ? 0xffffffffu : 0u;
            }
            F(k, kF_U2, t) = u * 0x00010001u;
            F(k, kF_CM, t) = (128u - m1) * kB1;
            F(k, kF_D2, t) = d2;
        }
    }

    __device__ void count(const DevNet &net, const int8_t *x, int t, bool cg)
    {
        block_count(net, x, t, out_nz, pos_in, cg);
    }

    __device__ void change_edge(const DevNet &net, int t, int owner, int pos, int w, int p, int tt)
    {
        if (t != owner) return;
        const int row = lut_row(net, (pos >> 8) & 0xff, pos & 0xff);
        const uint32_t a = (uint32_t)(row * kBT + t);
        undo_lut = true;
        undo_addr = a;
        undo_val = lut[a];
        lut[a] = edge_word_s(w, p, tt, undo_val);
    }

    __device__ void change_node(int t, int owner, int k, int kind, int v)
    {
        if (t != owner) return;
        const int f = kind == 3 ? kF_U2 : kind == 4 ? kF_CM : kF_D2;
        const uint32_t a = (uint32_t)((k * kF_N + f) * kBT + t);
        undo_lut = false;
        undo_addr = a;
        undo_val = node[a];
        node[a] = kind == 3 ? (uint32_t)v * 0x00010001u
                : kind == 4 ? (127u - (uint32_t)v) * kB1
                            : (v == 2 ? 0xffffffffu : 0u);
    }

    __device__ void undo(int t, int owner)
    {
        if (t != owner) return;
        if (undo_lut) lut[undo_addr] = undo_val;
        else node[undo_addr] = undo_val;
    }

    // Simulate(x) of Table 1 over every condition and time step, scored
    // against the entry tables (Section 2.3).  Returns y in every thread.
    __device__ int32_t simulate(const DevNet &net, int t, uint8_t *traj)
    {
        const int T = net.T, lane = t & 31, warp = t >> 5;
        uint32_t score = 0;
        for (int g = 0; g < net.G; ++g) {
            for (int k = 0; k < npl; ++k) {
                const size_t q = (size_t)g * kBT * npl + t * npl + k;
                const uint32_t s4 = __ldg(net.init_s4 + q);
                F(k, kF_S4, t) = s4;
                F(k, kF_CU, t) = 0;
                F(k, kF_CD, t) = 0;
                F(k, kF_UA01, t) = F(k, kF_U2, t);
                F(k, kF_UA23, t) = F(k, kF_U2, t);
                F(k, kF_MOV, t) = __ldg(net.movable + q);
                code[t * npl + k] = SmemPath::code_of(s4);
            }
            __syncthreads();
            const int ncg = min(net.C - 4 * g, 4);
            for (int tau = 0; tau < T; ++tau) {
                if (tau > 0) {
                    if (net.async) {   // only the step's selected node may move
                        const uint32_t *mt = net.movable_t + ((size_t)(g * T + tau) * kBT + t) * npl;
                        for (int k = 0; k < npl; ++k) F(k, kF_MOV, t) = __ldg(mt + k);
                    }
                    uint32_t m01 = 0, m23 = 0;
                    int o = 0;
                    for (int k = 0; k < npl; ++k) {
                        const int D4 = groups4(net.D[k]);
                        const uint32_t acc = gather_rows<kBT>(lut + o * kBT + t, D4, sm);
                        o += D4;
                        const uint32_t s4 = F(k, kF_S4, t);
                        const uint32_t tgt = target4(acc);
                        const uint32_t dp = tgt + 2 * kB1 - s4;
                        const uint32_t up = (dp + 0x7D7D7D7Du) & kH;
                        const uint32_t dn = ~(dp + 0x7E7E7E7Eu) & kH;
                        const uint32_t cu = (F(k, kF_CU, t) + kB1) & prmt(up, 0u, 0xBA98u);
                        const uint32_t cd = (F(k, kF_CD, t) + kB1) & prmt(dn, 0u, 0xBA98u);
                        F(k, kF_CU, t) = cu;
                        F(k, kF_CD, t) = cd;
                        const uint32_t cm = F(k, kF_CM, t);
                        const uint32_t el = ((cu + cm) | (cd + cm)) & F(k, kF_MOV, t);
                        const uint32_t d2 = F(k, kF_D2, t);
                        const uint32_t step1 = s4 + (up >> 7) - (dn >> 7);
                        F(k, kF_SN, t) = (tgt & d2) | (step1 & ~d2);
                        F(k, kF_ELM, t) = prmt(el, 0u, 0xBA98u);
                        const uint32_t p01 = F(k, kF_UA01, t) & prmt(el, 0u, 0x9988u);
                        const uint32_t p23 = F(k, kF_UA23, t) & prmt(el, 0u, 0xBBAAu);
                        F(k, kF_PR01, t) = p01;
                        F(k, kF_PR23, t) = p23;
                        m01 = max_u16x2(m01, p01);
                        m23 = max_u16x2(m23, p23);
                    }
                    const uint32_t p0 = __reduce_max_sync(kFull, m01 & 0xffffu);
                    const uint32_t p1 = __reduce_max_sync(kFull, m01 >> 16);
                    const uint32_t p2 = __reduce_max_sync(kFull, m23 & 0xffffu);
                    const uint32_t p3 = __reduce_max_sync(kFull, m23 >> 16);
                    if (lane == 0) {
                        bc->wmax[warp][0] = p0;
                        bc->wmax[warp][1] = p1;
                        bc->wmax[warp][2] = p2;
                        bc->wmax[warp][3] = p3;
                    }
                    __syncthreads();
                    uint32_t q0 = 0, q1 = 0, q2 = 0, q3 = 0;
#pragma unroll
                    for (int w = 0; w < kBW; ++w) {
                        q0 = max(q0, bc->wmax[w][0]);
                        q1 = max(q1, bc->wmax[w][1]);
                        q2 = max(q2, bc->wmax[w][2]);
                        q3 = max(q3, bc->wmax[w][3]);
                    }
                    const uint32_t P01 = prmt(q0, q1, 0x5410u), P23 = prmt(q2, q3, 0x5410u);
                    for (int k = 0; k < npl; ++k) {
                        const uint32_t nz01 = ((F(k, kF_PR01, t) ^ P01) + 0x7FFF7FFFu) & 0x80008000u;
                        const uint32_t nz23 = ((F(k, kF_PR23, t) ^ P23) + 0x7FFF7FFFu) & 0x80008000u;
                        const uint32_t upd = F(k, kF_ELM, t) & ~prmt(nz01, nz23, 0xFDB9u);
                        const uint32_t s4 = (F(k, kF_S4, t) & ~upd) | (F(k, kF_SN, t) & upd);
                        F(k, kF_S4, t) = s4;
                        F(k, kF_CU, t) &= ~upd;
                        F(k, kF_CD, t) &= ~upd;
                        const uint32_t u2 = F(k, kF_U2, t);
                        const uint32_t u01 = prmt(upd, 0u, 0x9988u), u23 = prmt(upd, 0u, 0xBBAAu);
                        F(k, kF_UA01, t) = ((F(k, kF_UA01, t) + u2) & ~u01) | (u2 & u01);
                        F(k, kF_UA23, t) = ((F(k, kF_UA23, t) + u2) & ~u23) | (u2 & u23);
                        code[t * npl + k] = SmemPath::code_of(s4);
                    }
                    __syncthreads();
                }
                // error at this time point (compact entry words)
                const uint32_t *ob = net.obs + (((size_t)g * T + tau) * kBT + t) * npl;
                for (int k = 0; k < npl; ++k) {
                    const uint32_t s4 = F(k, kF_S4, t);
                    score = entry_error(s4, __ldg(ob + k), score);
                    if (traj) {
                        const int i = net.q_node[t * npl + k];
                        for (int c = 0; c < ncg; ++c)
                            if (i >= 0)
                                traj[((size_t)(4 * g + c) * T + tau) * net.N + i] =
                                    (uint8_t)((s4 >> (8 * c)) & 0xffu);
                    }
                }
            }
            __syncthreads();
        }
        score = __reduce_add_sync(kFull, score);
        if (lane == 0) bc->wsum[warp] = score;
        __syncthreads();
        uint32_t total = 0;
#pragma unroll
        for (int w = 0; w < kBW; ++w) total += bc->wsum[w];
        __syncthreads();
        return (int32_t)(total >> 2);   // quarter units (entry_error)
    }
};

__device__ __forceinline__ BlockPath make_block_path(const DevNet &net, uint8_t *sm)
{
    const BlockLayout L = block_layout(net.D, net.npl, net.N);
    BlockPath P;
    P.sm = sm;
    P.code = reinterpret_cast<uint16_t *>(sm + L.codes);
    P.lut = reinterpret_cast<uint32_t *>(sm + L.lut);
    P.node = reinterpret_cast<uint32_t *>(sm + L.node);
    P.out_nz = sm + L.cnt;
    P.pos_in = P.out_nz + ((net.N + 15) & ~15);
    P.bc = reinterpret_cast<Bcast *>(sm + L.scratch);
    P.xs = reinterpret_cast<int8_t *>(sm + L.x);
    P.npl = net.npl;
    return P;
}

// Block-wide reductions and barriers for simulate_swar4_core: warp redux, then
// the eight warp values through the broadcast area.  A time point's compact
// entry words (one per node, 4 conditions) are loaded at the start of its
// update step, so that their latency overlaps the gather, the update and its
// barriers (all warps of the block would otherwise wait on L2 at once).
template <int NPL>
struct BlockSync {
    Bcast *bc;
    int lane, warp;
    uint32_t *codes2;   // the second copy of the codes (code_word2), or null

    struct Ahead {
        uint32_t w[NPL];
    };
    template <int>
    __device__ __forceinline__ Ahead fetch_obs(const DevNet &net, int g, int tau, int t) const
    {
        Ahead a;
        load_obs<NPL>(a.w, net.obs + (((size_t)g * net.T + tau) * kBT + t) * NPL);
        return a;
    }
    template <int, bool>
    __device__ __forceinline__ uint32_t error(const Ahead &a, const uint32_t (&s4)[NPL],
                                              const DevNet &, int, int, int, int) const
    {
        uint32_t e = 0;
#pragma unroll
        for (int k = 0; k < NPL; ++k) e = entry_error(s4[k], a.w[k], e);
        return e;
    }

    __device__ __forceinline__ void max4(uint32_t m01, uint32_t m23, uint32_t &P01,
                                         uint32_t &P23) const
    {
        const uint32_t p0 = __reduce_max_sync(kFull, m01 & 0xffffu);
        const uint32_t p1 = __reduce_max_sync(kFull, m01 >> 16);
        const uint32_t p2 = __reduce_max_sync(kFull, m23 & 0xffffu);
        const uint32_t p3 = __reduce_max_sync(kFull, m23 >> 16);
        if (lane == 0)
            *reinterpret_cast<uint4 *>(bc->wmax[warp]) = make_uint4(p0, p1, p2, p3);
        __syncthreads();
        uint4 q = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int w = 0; w < kBW; ++w) {
            const uint4 v = *reinterpret_cast<const uint4 *>(bc->wmax[w]);
            q.x = max(q.x, v.x);
            q.y = max(q.y, v.y);
            q.z = max(q.z, v.z);
            q.w = max(q.w, v.w);
        }
        P01 = prmt(q.x, q.y, 0x5410u);
        P23 = prmt(q.z, q.w, 0x5410u);
    }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ uint32_t sum(uint32_t v) const
    {
        v = __reduce_add_sync(kFull, v);
        if (lane == 0) bc->wsum[warp] = v;
        __syncthreads();
        uint32_t total = 0;
#pragma unroll
        for (int w = 0; w < kBW; ++w) total += bc->wsum[w];
        __syncthreads();
        return total;
    }
    // Both copies of the thread's state codes: its NPL / 2 words at p (the
    // first copy) and each word w = t NPL / 2 + j at code_word2(w) of the
    // second (for 2, 4 and 8 nodes per thread a warp's stores of one j fall
    // in 32 distinct banks).
    template <int, bool SMEM_FMT>
    __device__ __forceinline__ void store_codes(uint8_t *p, const uint32_t (&s4)[NPL], int t) const
    {
        static_assert(NPL % 2 == 0, "codes are stored in pairs");
        uint32_t w[NPL / 2];
#pragma unroll
        for (int j = 0; j < NPL / 2; ++j) w[j] = state_code_pair<SMEM_FMT>(s4[2 * j], s4[2 * j + 1]);
        if constexpr (NPL == 2) {
            *reinterpret_cast<uint32_t *>(p) = w[0];
        } else if constexpr (NPL == 4) {
            *reinterpret_cast<uint2 *>(p) = make_uint2(w[0], w[1]);
        } else if constexpr (NPL == 8) {
            *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
#pragma unroll
            for (int j = 0; j < NPL / 2; ++j) reinterpret_cast<uint32_t *>(p)[j] = w[j];
        }
        if (codes2) {
#pragma unroll
            for (int j = 0; j < NPL / 2; ++j)
                codes2[code_word2((uint32_t)(t * (NPL / 2) + j))] = w[j];
        }
    }
};

// Register variant for 2, 4, 6 or 8 nodes per thread (513 .. 2048 nodes, and
// the small networks of high in-degree): the table rows stay in shared memory
// as above, while each thread keeps its nodes' parameters and byte-SIMD update
// state in registers (the warp paths' simulate_swar4_core, with block-wide
// maxima), so that an update step touches shared memory only in the gather
// and the state codes.
template <int NPL>
struct BlockRegPath {
    uint8_t *sm;
    uint32_t *lut;
    uint8_t *out_nz, *pos_in;
    Bcast *bc;
    int8_t *xs;   // the chain's x in shared memory (when the launch reserved it)
    static constexpr int npl = NPL;
    uint32_t codes2;   // byte offset of the second copy of the codes (0: none)
    int32_t u[NPL], m1[NPL], d2[NPL];
    uint32_t undo_addr, undo_val;
    int undo_kind, undo_slot;

    __device__ __forceinline__ int lut_row(const DevNet &net, int k, int d) const
    {
        int o = 0;
        for (int kk = 0; kk < k; ++kk) o += groups4(net.D[kk]);
        return o + d;
    }

    __device__ void load(const DevNet &net, const int8_t *x, int t, bool cg)
    {
        auto X = [&](int j) { return cg ? xcg(x, j) : (int)x[j]; };
        const int E = net.E, N = net.N;
        int o = 0;
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
            for (int d = 0; d < net.D[k]; ++d) {
                const int v = net.edge_id[(k * net.dtab + d) * kBT + t];
                uint32_t w = 0x04040000u | ((uint32_t)(-1 - v) & 0xffffu);   // padding
                if (v >= 0) {
                    // the source's code in the copy the layout chose for this entry
                    const int e = v & ~kCodeCopy2;
                    const uint32_t q = (uint32_t)net.node_q[net.src[e]];
                    const uint32_t a = (v & kCodeCopy2)
                                           ? codes2 + 4u * code_word2(q >> 1) + 2u * (q & 1u)
                                           : 2u * q;
                    w = edge_word_s(X(e), X(E + e), X(2 * E + e), a);
                }
                lut[(o + d) * kBT + t] = w;
            }
            // neutral rows up to a whole group of 4: the code of node 2 t
            for (int d = net.D[k]; d < groups4(net.D[k]); ++d)
                lut[(o + d) * kBT + t] = 0x04040000u | (4u * (uint32_t)t);
            o += groups4(net.D[k]);
            const int i = net.q_node[t * NPL + k];
            u[k] = i >= 0 ? (net.sync ? 0 : X(3 * E + i)) : 1;
            m1[k] = i >= 0 ? X(3 * E + N + i) + 1 : 1;
            d2[k] = i >= 0 ? X(3 * E + 2 * N + i) == 2 : 0;
        }
    }

    __device__ void count(const DevNet &net, const int8_t *x, int t, bool cg)
    {
        block_count(net, x, t, out_nz, pos_in, cg);
    }

    __device__ void change_edge(const DevNet &net, int t, int owner, int pos, int w, int p, int tt)
    {
        if (t != owner) return;
        const uint32_t a = (uint32_t)(lut_row(net, (pos >> 8) & 0xff, pos & 0xff) * kBT + t);
        undo_kind = 0;
        undo_addr = a;
        undo_val = lut[a];
        lut[a] = edge_word_s(w, p, tt, undo_val);
    }

    __device__ void change_node(int t, int owner, int slot, int kind, int v)
    {
        if (t != owner) return;
        undo_kind = kind;
        undo_slot = slot;
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
            if (k != slot) continue;
            if (kind == 3) { undo_val = (uint32_t)u[k]; u[k] = v; }
            else if (kind == 4) { undo_val = (uint32_t)m1[k]; m1[k] = v + 1; }
            else { undo_val = (uint32_t)d2[k]; d2[k] = v == 2; }
        }
    }

    __device__ void undo(int t, int owner)
    {
        if (t != owner) return;
        if (undo_kind == 0) {
            lut[undo_addr] = undo_val;
            return;
        }
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
            if (k != undo_slot) continue;
            if (undo_kind == 3) u[k] = (int32_t)undo_val;
            else if (undo_kind == 4) m1[k] = (int32_t)undo_val;
            else d2[k] = (int32_t)undo_val;
        }
    }

    // Simulate(x) of Table 1 (Sections 2.1-2.3); y in every thread.
    __device__ int32_t simulate(const DevNet &net, int t, uint8_t *traj)
    {
        SlotGather<NPL, kBT, true> gather;
        gather.lut = lut + t;
        gather.sm = sm;
        int o = 0;
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
            gather.row0[k] = o;
            // this warp's rows of the slot (its edges come first)
            gather.d4[k] = __ldg(net.warp_d4 + k * (kBT / 32) + (t >> 5));
            o += groups4(net.D[k]);
        }
        const BlockSync<NPL> sync{bc, t & 31, t >> 5,
                                  codes2 ? reinterpret_cast<uint32_t *>(sm + codes2) : nullptr};
        return simulate_swar4_core<NPL, true, false, kBT>(u, m1, d2, net, sm, 0u, t, traj,
                                                          INT32_MAX, gather, sync);
    }
};

template <int NPL>
__device__ __forceinline__ BlockRegPath<NPL> make_block_reg_path(const DevNet &net, uint8_t *sm)
{
    const BlockLayout L = block_layout(net.D, NPL, net.N);
    BlockRegPath<NPL> P;
    P.sm = sm;
    P.codes2 = L.codes2;
    P.lut = reinterpret_cast<uint32_t *>(sm + L.lut);
    P.out_nz = sm + L.cnt;
    P.pos_in = P.out_nz + ((net.N + 15) & ~15);
    P.bc = reinterpret_cast<Bcast *>(sm + L.scratch);
    P.xs = reinterpret_cast<int8_t *>(sm + L.x);
    return P;
}

// make_path<Path>: the shared-memory layout of either variant.
template <class Path> struct PathMaker;
template <> struct PathMaker<BlockPath> {
    static __device__ __forceinline__ BlockPath make(const DevNet &net, uint8_t *sm)
    {
        return make_block_path(net, sm);
    }
};
template <int NPL> struct PathMaker<BlockRegPath<NPL>> {
    static __device__ __forceinline__ BlockRegPath<NPL> make(const DevNet &net, uint8_t *sm)
    {
        return make_block_reg_path<NPL>(net, sm);
    }
};

template <class Path>
__global__ void __launch_bounds__(kBT, 1)
    evaluate_block_kernel(DevNet net, const int8_t *__restrict__ X, int64_t xstride, int32_t n,
                          int32_t *__restrict__ score, int32_t *__restrict__ score2,
                          uint8_t *__restrict__ traj)
{
    extern __shared__ __align__(256) uint8_t sm[];
    Path P = PathMaker<Path>::make(net, sm);
    const int t = threadIdx.x;
    for (int v = blockIdx.x; v < n; v += gridDim.x) {
        P.load(net, X + (size_t)v * xstride, t, false);
        __syncthreads();
        uint8_t *tv = traj ? traj + (size_t)v * net.C * net.T * net.N : nullptr;
        const int32_t y = P.simulate(net, t, tv);
        if (t == 0) {
            score[v] = y;
            if (score2) score2[v] = y;
        }
        __syncthreads();
    }
}

// Copy a row of `bytes` (a multiple of 16) block-wide; a global side is read
// or written through L2 (another SM may run the chain's next chunk).
template <bool SRC_GLOBAL, bool DST_GLOBAL>
__device__ __forceinline__ void block_copy16(int8_t *dst, const int8_t *src, int bytes, int t)
{
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    for (int k = t; k < (bytes >> 4); k += kBT) {
        const uint4 v = SRC_GLOBAL ? __ldcg(s + k) : s[k];
        if (DST_GLOBAL) __stcg(d + k, v);
        else d[k] = v;
    }
}

// Steps [g_lo, g_hi) of one chain (Table 1), then publish the chunk.  With XS
// the chain's x is copied into shared memory for the chunk (one coalesced row
// instead of scattered L2 reads by the table build, the constraint counters and
// the proposals) and written back at its end.
template <class Path, bool XS>
__device__ void block_chunk(Path &P, const DevNet &net, const DevChains &ch,
                            const DevSched &sc, int chain, int64_t g_lo, int64_t g_hi,
                            int done_value, int t)
{
    const int E = net.E;
    int8_t *xg = ch.x_cur + (size_t)chain * ch.pstride;
    int8_t *xb = ch.x_best + (size_t)chain * ch.pstride;
    int8_t *xr = xg;   // where x is read and written during the chunk
    if constexpr (XS) {
        xr = P.xs;
        block_copy16<true, false>(xr, xg, ch.pstride, t);
        __syncthreads();
    }
    Bcast *bc = P.bc;
    P.load(net, xr, t, !XS);
    P.count(net, xr, t, !XS);
    __syncthreads();
    int32_t d_cur = __ldcg(ch.d_cur + chain), d_best = __ldcg(ch.d_best + chain);
    int32_t n_acc = 0, n_up = 0, n_null = 0;
    int64_t level = g_lo / sc.iters;
    int64_t in_level = g_lo - level * sc.iters;
    auto X = [&](int j) { return XS ? (int)xr[j] : xcg(xg, j); };
    for (int64_t g = g_lo; g < g_hi; ++g) {
        if (in_level == sc.iters) {
            in_level = 0;
            ++level;
        }
        if (sc.reset_to_best && in_level == 0) {
            // Table 1: every level starts from the chain's x_best
            block_copy16<true, !XS>(xr, xb, ch.pstride, t);
            __threadfence_block();
            __syncthreads();
            P.load(net, xr, t, !XS);
            P.count(net, xr, t, !XS);
            __syncthreads();
            d_cur = d_best;
        }
        ++in_level;
        if (t == 0) {
            const uint4 r = philox(ch.seed, (uint32_t)g, (uint32_t)((uint64_t)g >> 32),
                                   (uint32_t)chain, 0u);
            int j = 0, kind = 0, idx = 0, cur = 0, v = 0;
            const bool ok = net.n_free > 0 &&
                            get_candidate_x(net, X, P.out_nz, P.pos_in, r.x, r.y, j, kind, idx,
                                            cur, v);
            bc->ok = ok;
            if (ok) {
                bc->j = j;
                bc->kind = kind;
                bc->idx = idx;
                bc->cur = cur;
                bc->v = v;
                bc->rz = r.z;
                if (kind < 3) {
                    const int pos = net.edge_pos[idx];
                    int w = X(idx), p = X(E + idx), tt = X(2 * E + idx);
                    if (kind == 0) w = v; else if (kind == 1) p = v; else tt = v;
                    bc->owner = pos >> 16;
                    bc->pos = pos;
                    bc->w = w;
                    bc->p = p;
                    bc->t = tt;
                } else {
                    const int q = net.node_q[idx];
                    bc->owner = q / P.npl;
                    bc->slot = q - (q / P.npl) * P.npl;
                }
            }
        }
        __syncthreads();
        if (!bc->ok) {
            ++n_null;
            __syncthreads();
            continue;
        }
        const int owner = bc->owner, kind = bc->kind;
        if (kind < 3) P.change_edge(net, t, owner, bc->pos, bc->w, bc->p, bc->t);
        else P.change_node(t, owner, bc->slot, kind, bc->v);
        const int j = bc->j, v = bc->v, cur = bc->cur, idx = bc->idx;
        const uint32_t rz = bc->rz;
        __syncthreads();
        const int32_t d_cand = P.simulate(net, t, nullptr);
        // Metropolis acceptance against the host-computed threshold table
        const int32_t dE = d_cand - d_cur;
        bool accept = dE <= 0;
        if (!accept) {
            const int64_t l = level - sc.level0;
            if (dE <= sc.thr_len[l]) accept = rz < __ldg(sc.thr + sc.thr_off[l] + dE - 1);
        }
        if (accept) {
            if (t == 0) {
                apply_counters_x(net, X, P.out_nz, P.pos_in, kind, idx, cur, v);
                if (XS) xr[j] = (int8_t)v;
                else __stcg(xg + j, (int8_t)v);
            }
            d_cur = d_cand;
            ++n_acc;
            n_up += dE > 0;
            __syncthreads();
            if (d_cand < d_best) {
                d_best = d_cand;
                block_copy16<!XS, true>(xb, xr, ch.pstride, t);
            }
        } else {
            P.undo(t, owner);
        }
        __syncthreads();
    }
    if (t == 0) {
        __stcg(ch.d_cur + chain, d_cur);
        __stcg(ch.d_best + chain, d_best);
        int64_t *cnt = ch.cnt + 3 * (size_t)chain;
        __stcg(cnt + 0, __ldcg(cnt + 0) + n_acc);
        __stcg(cnt + 1, __ldcg(cnt + 1) + n_up);
        __stcg(cnt + 2, __ldcg(cnt + 2) + n_null);
    }
    if constexpr (XS) block_copy16<false, true>(xg, xr, ch.pstride, t);
    // publish: every thread's stores, then the chunk counter of the chain
    __threadfence();
    __syncthreads();
    if (t == 0) atomicExch(sc.done + chain, done_value);
}

// Thread 0 waits (bounded) until chunk cj - 1 of the chain is published.
__device__ __forceinline__ bool block_wait(int32_t *flag, int cj, int32_t *err)
{
    for (int k = 0; k < kWaitLimit; ++k) {
        if (*(volatile int32_t *)err) return false;
        if (atomicAdd(flag, 0) >= cj) {
            __threadfence();
            return true;
        }
        __nanosleep(256);
    }
    atomicExch(err, 1);
    return false;
}

template <class Path, bool XS>
__global__ void __launch_bounds__(kBT, 1) anneal_block_kernel(DevNet net, DevChains ch, DevSched sc)
{
    extern __shared__ __align__(256) uint8_t sm[];
    Path P = PathMaker<Path>::make(net, sm);
    const int t = threadIdx.x;
    const int64_t n_items = (int64_t)sc.n_chunks * ch.n;
    for (;;) {
        if (t == 0) P.bc->item = atomicAdd(sc.queue, 1u);
        __syncthreads();
        const unsigned int item = P.bc->item;
        __syncthreads();
        if ((int64_t)item >= n_items) break;
        const int cj = (int)(item / (unsigned)ch.n);
        const int chain = (int)(item - (unsigned)cj * (unsigned)ch.n);
        if (cj > 0) {
            if (t == 0) P.bc->ok = block_wait(sc.done + chain, cj, sc.err);
            __syncthreads();
            const bool ok = P.bc->ok;
            __syncthreads();
            if (!ok) return;
        }
        const int64_t g_lo = sc.g0 + (int64_t)cj * sc.chunk;
        const int64_t g_hi = min(sc.g1, g_lo + sc.chunk);
        block_chunk<Path, XS>(P, net, ch, sc, chain, g_lo, g_hi, cj + 1, t);
    }
}

// Finish of a screened step (the learned proposal screen) for block-path
// networks, a block per chain: warp 0 selects the moves to simulate (as the
// warp paths do), each is simulated exactly on the chain's tables (change,
// Simulate, undo), and the one of lowest exact score (first on ties) goes to
// the Metropolis test of Table 1; an accepted move updates x_cur, delta_cur,
// the best vector (strict improvement), the counters and A1.
template <class Path, bool XS>
__global__ void __launch_bounds__(kBT, 1) screen_finish_block_kernel(ScreenArgs a, DevSched sc)
{
    extern __shared__ __align__(256) uint8_t sm[];
    const DevNet &net = a.net;
    Path P = PathMaker<Path>::make(net, sm);
    Bcast *bc = P.bc;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int E = net.E, N = net.N;
    for (int c = blockIdx.x; c < a.ch.n; c += gridDim.x) {
        const uint4 r = step_draw(a.ch, a.g, c, 0u);
        if (warp == 0) {
            int chosen[kMaxTop];
            select_candidates(a, c, lane, r, chosen);
            if (lane == 0)
                for (int s = 0; s < kMaxTop; ++s) bc->sel[s] = chosen[s];
        }
        __syncthreads();
        int chosen[kMaxTop];
#pragma unroll
        for (int s = 0; s < kMaxTop; ++s) chosen[s] = bc->sel[s];
        int64_t *cnt = a.ch.cnt + 3 * (size_t)c;
        if (chosen[0] < 0) {
            if (t == 0) cnt[2] += 1;
            __syncthreads();
            continue;
        }
        int8_t *xg = a.ch.x_cur + (size_t)c * a.ch.pstride;
        int8_t *xr = xg;
        if constexpr (XS) {
            xr = P.xs;
            block_copy16<true, false>(xr, xg, a.ch.pstride, t);
            __syncthreads();
        }
        P.load(net, xr, t, false);
        __syncthreads();
        int best = -1;
        int32_t d = 0;
#pragma unroll
        for (int s = 0; s < kMaxTop; ++s) {
            const int move = chosen[s];
            if (move < 0) continue;
            const int j = move >> 8, v = (int8_t)(move & 255);
            int kind, idx, owner;
            param_kind(j, E, N, kind, idx);
            if (kind < 3) {
                const int pos = net.edge_pos[idx];
                owner = pos >> 16;
                int w = xr[idx], p = xr[E + idx], tt = xr[2 * E + idx];
                if (kind == 0) w = v; else if (kind == 1) p = v; else tt = v;
                P.change_edge(net, t, owner, pos, w, p, tt);
            } else {
                const int q = net.node_q[idx];
                owner = q / P.npl;
                P.change_node(t, owner, q - owner * P.npl, kind, v);
            }
            __syncthreads();
            const int32_t ds = P.simulate(net, t, nullptr);
            P.undo(t, owner);
            __syncthreads();
            if (best < 0 || ds < d) { best = move; d = ds; }
        }
        const int32_t d_cur = a.ch.d_cur[c], d_best = a.ch.d_best[c];
        const int32_t dE = d - d_cur;
        bool accept = dE <= 0;
        if (!accept) {
            const int64_t l = a.g / sc.iters - sc.level0;
            if (dE <= sc.thr_len[l]) accept = r.z < __ldg(sc.thr + sc.thr_off[l] + dE - 1);
        }
        if (accept) {
            const int j = best >> 8, v = (int8_t)(best & 255);
            const int rn = a.row_base[j] + v, ro = a.row_base[j] + xr[j];
            __syncthreads();
            if (t == 0) {
                xg[j] = (int8_t)v;
                a.ch.d_cur[c] = d;
                cnt[0] += 1;
                cnt[1] += dE > 0;
            }
            __syncthreads();
            if (d < d_best) {
                block_copy16<true, true>(a.ch.x_best + (size_t)c * a.ch.pstride, xg, a.ch.pstride, t);
                if (t == 0) a.ch.d_best[c] = d;
            }
            for (int h = t; h < a.H1; h += kBT)
                a.A1[(size_t)c * a.H1 + h] += __bfloat162float(a.W1b[(size_t)rn * a.H1 + h]) -
                                              __bfloat162float(a.W1b[(size_t)ro * a.H1 + h]);
        }
        __syncthreads();
    }
}

cudaError_t smem_limit(int *limit)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return e;
}

cudaError_t block_smem(const DevNet &net, size_t *bytes)
{
    *bytes = block_layout(net.D, net.npl, net.N).bytes;
    int limit = 0;
    cudaError_t e = smem_limit(&limit);
    if (e != cudaSuccess) return e;
    return *bytes <= (size_t)limit ? cudaSuccess : cudaErrorInvalidConfiguration;
}

}  // namespace

size_t block_path_smem_bytes(const int *D, int npl, int N)
{
    return block_layout(D, npl, N).bytes;
}

bool block_path_two_copies(const int *D, int npl, int N)
{
    return block_layout(D, npl, N).codes2 != 0;
}

namespace {

template <class Path>
cudaError_t evaluate_block_t(const DevNet &net, const int8_t *X, int64_t xstride, int32_t n,
                             int32_t *score, int32_t *score2, uint8_t *traj, int sm_count,
                             cudaStream_t st)
{
    size_t smem = 0;
    cudaError_t e = block_smem(net, &smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(evaluate_block_kernel<Path>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, evaluate_block_kernel<Path>, kBT,
                                                      smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t cap = (int64_t)sm_count * per_sm;
    const int grid = (int)(n < cap ? n : cap);
    evaluate_block_kernel<Path><<<grid, kBT, smem, st>>>(net, X, xstride, n, score, score2, traj);
    return cudaGetLastError();
}

template <class Path, bool XS>
cudaError_t anneal_block_launch(const DevNet &net, const DevChains &ch, const DevSched &sc0,
                                size_t smem, int sm_count, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(anneal_block_kernel<Path, XS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, anneal_block_kernel<Path, XS>,
                                                      kBT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = sm_count * per_sm;
    DevSched sc = sc0;
    plan_chunks(sc, ch.n, grid);
    e = cudaMemsetAsync(sc.queue, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc.done, 0, sizeof(int32_t) * (size_t)ch.n, st);
    if (e != cudaSuccess) return e;
    anneal_block_kernel<Path, XS><<<grid, kBT, smem, st>>>(net, ch, sc);
    return cudaGetLastError();
}

// The chain's x is kept in shared memory where it fits beside the tables.
template <class Path>
cudaError_t anneal_block_t(const DevNet &net, const DevChains &ch, const DevSched &sc0,
                           int sm_count, cudaStream_t st)
{
    size_t smem = 0;
    cudaError_t e = block_smem(net, &smem);
    if (e != cudaSuccess) return e;
    int limit = 0;
    if ((e = smem_limit(&limit)) != cudaSuccess) return e;
    const size_t with_x = block_layout(net.D, net.npl, net.N, (uint32_t)ch.pstride).bytes;
    if (with_x <= (size_t)limit)
        return anneal_block_launch<Path, true>(net, ch, sc0, with_x, sm_count, st);
    return anneal_block_launch<Path, false>(net, ch, sc0, smem, sm_count, st);
}

template <class Path, bool XS>
cudaError_t finish_block_launch(const ScreenArgs &a, const DevSched &sc, size_t smem,
                                int sm_count, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(screen_finish_block_kernel<Path, XS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, screen_finish_block_kernel<Path, XS>,
                                                      kBT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t cap = (int64_t)sm_count * per_sm;
    const int grid = (int)(a.ch.n < cap ? a.ch.n : cap);
    screen_finish_block_kernel<Path, XS><<<grid, kBT, smem, st>>>(a, sc);
    return cudaGetLastError();
}

template <class Path>
cudaError_t finish_block_t(const ScreenArgs &a, const DevSched &sc, int sm_count, cudaStream_t st)
{
    size_t smem = 0;
    cudaError_t e = block_smem(a.net, &smem);
    if (e != cudaSuccess) return e;
    int limit = 0;
    if ((e = smem_limit(&limit)) != cudaSuccess) return e;
    const size_t with_x = block_layout(a.net.D, a.net.npl, a.net.N, (uint32_t)a.ch.pstride).bytes;
    if (with_x <= (size_t)limit) return finish_block_launch<Path, true>(a, sc, with_x, sm_count, st);
    return finish_block_launch<Path, false>(a, sc, smem, sm_count, st);
}

}  // namespace

cudaError_t launch_finish_block(const ScreenArgs &a, const DevSched &sc, int sm_count,
                                cudaStream_t st)
{
    switch (a.net.npl) {
    case 2: return finish_block_t<BlockRegPath<2>>(a, sc, sm_count, st);
    case 4: return finish_block_t<BlockRegPath<4>>(a, sc, sm_count, st);
    case 6: return finish_block_t<BlockRegPath<6>>(a, sc, sm_count, st);
    case 8: return finish_block_t<BlockRegPath<8>>(a, sc, sm_count, st);
    default: return finish_block_t<BlockPath>(a, sc, sm_count, st);
    }
}

cudaError_t launch_evaluate_block(const DevNet &net, const int8_t *X, int64_t xstride, int32_t n,
                                  int32_t *score, int32_t *score2, uint8_t *traj, int sm_count,
                                  cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    switch (net.npl) {
    case 2: return evaluate_block_t<BlockRegPath<2>>(net, X, xstride, n, score, score2, traj, sm_count, st);
    case 4: return evaluate_block_t<BlockRegPath<4>>(net, X, xstride, n, score, score2, traj, sm_count, st);
    case 6: return evaluate_block_t<BlockRegPath<6>>(net, X, xstride, n, score, score2, traj, sm_count, st);
    case 8: return evaluate_block_t<BlockRegPath<8>>(net, X, xstride, n, score, score2, traj, sm_count, st);
    default: return evaluate_block_t<BlockPath>(net, X, xstride, n, score, score2, traj, sm_count, st);
    }
}

cudaError_t launch_anneal_block(const DevNet &net, const DevChains &ch, const DevSched &sc0,
                                int sm_count, cudaStream_t st)
{
    switch (net.npl) {
    case 2: return anneal_block_t<BlockRegPath<2>>(net, ch, sc0, sm_count, st);
    case 4: return anneal_block_t<BlockRegPath<4>>(net, ch, sc0, sm_count, st);
    case 6: return anneal_block_t<BlockRegPath<6>>(net, ch, sc0, sm_count, st);
    case 8: return anneal_block_t<BlockRegPath<8>>(net, ch, sc0, sm_count, st);
    default: return anneal_block_t<BlockPath>(net, ch, sc0, sm_count, st);
    }
}

}  // namespace rn
