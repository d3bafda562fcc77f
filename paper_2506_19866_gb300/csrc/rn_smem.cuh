// rn_smem.cuh -- the shared-memory-table simulator: any number of nodes per
// lane up to 16 (N <= 512), chosen at run time.
//
// Same warp-per-chain scheme and byte-SIMD update as the register kernels
// (rn_device.cuh), but the per-chain in-edge table words and the per-node
// update state live in the warp's shared memory instead of registers, laid
// out [..][lane] so that every access of the warp is one conflict-free
// wavefront.  Table word of an edge:
//
//   bytes 0-1  shared-memory offset of the source's 16-bit state code
//   byte 2     4 + (2 // t) * w * p
//   byte 3     4 + (1 // t) * w * p
//
// and the state code of a node holds 4 - s_c in nibble c, so that PRMT against
// 0x04040404 reads the constant 4 (state 0, no input), byte 3 (state 1) or
// byte 2 (state 2) for every condition of the group at once (Section 2.1).
#pragma once

#include "rn_device.cuh"

namespace rn {

// Per-node words in shared memory, [slot][field][lane].
enum : int {
    kF_S4 = 0,   // states (byte c = condition c)
    kF_CU,       // consecutive up drives
    kF_CD,       // consecutive down drives
    kF_UA01,     // u * age, conditions 0 and 1 (16-bit lanes)
    kF_UA23,     // u * age, conditions 2 and 3
    kF_MOV,      // bit 7 of byte c: may move in condition c
    kF_U2,       // u in both 16-bit lanes
    kF_CM,       // (128 - (m + 1)) in every byte
    kF_D2,       // all ones if d = 2
    kF_SN,       // candidate next states (between the two phases of a step)
    kF_PR01,     // eligible priorities, conditions 0 and 1
    kF_PR23,     // eligible priorities, conditions 2 and 3
    kF_ELM,      // eligible mask (byte per condition)
    kF_N
};

__host__ __device__ __forceinline__ uint32_t edge_word_s(int w, int p, int t, uint32_t addr)
{
    const int wp = w * p;
    const int f1 = (t == 1) ? wp : 0;
    const int f2 = (t == 1) ? 2 * wp : wp;
    return (addr & 0xffffu) | ((uint32_t)(4 + f2) << 16) | ((uint32_t)(4 + f1) << 24);
}

// Shared-memory footprint of one warp (bytes; multiple of 16) and of the
// code region that precedes all warp regions in the block (1 KiB per warp).
// Each slot's table has groups4(D_k) rows: the rows past D_k are neutral.
__host__ __device__ inline uint32_t smem_path_lut_words(const int *D, int npl)
{
    uint32_t s = 0;
    for (int k = 0; k < npl; ++k) s += (uint32_t)groups4(D[k]);
    return s * 32u;
}

__host__ __device__ inline uint32_t smem_path_warp_bytes(uint32_t lut_words, int npl, int pstride,
                                                         int N)
{
    const uint32_t node = (uint32_t)npl * kF_N * 32u * 4u;
    const uint32_t cnt = 2u * (((uint32_t)N + 15u) & ~15u);
    return lut_words * 4u + node + (uint32_t)pstride + cnt;
}

constexpr uint32_t kCodeBytesPerWarp = 1024u;   // 16-bit codes of up to 512 nodes

struct SmemPath {
    uint8_t *sm;         // dynamic shared memory of the block
    uint32_t codes;      // offset of this warp's code array in sm
    uint32_t *lut;       // [sum D_k][32]
    uint32_t *node;      // [npl][kF_N][32]
    int npl;
    // undo record of the owner lane
    uint32_t undo_addr;  // element index into lut or node
    uint32_t undo_val;
    bool undo_lut;

    __device__ __forceinline__ uint32_t &F(int k, int f, int lane) const
    {
        return node[(k * kF_N + f) * 32 + lane];
    }

    __device__ __forceinline__ int lut_row(const DevNet &net, int k, int d) const
    {
        int o = 0;
        for (int kk = 0; kk < k; ++kk) o += groups4(net.D[kk]);
        return o + d;
    }

    // Build the warp's tables from a parameter vector x.
    __device__ void load(const DevNet &net, const int8_t *x, int lane)
    {
        const int E = net.E, N = net.N;
        int o = 0;
        for (int k = 0; k < npl; ++k) {
            for (int d = 0; d < net.D[k]; ++d) {
                const int e = net.edge_id[(k * net.dtab + d) * 32 + lane];
                uint32_t w;
                if (e >= 0)
                    w = edge_word_s(x[e], x[E + e], x[2 * E + e],
                                    codes + 2u * (uint32_t)net.node_q[net.src[e]]);
                else
                    w = 0x04040000u | ((codes + (uint32_t)(-1 - e)) & 0xffffu);
                lut[(o + d) * 32 + lane] = w;
            }
            // neutral rows up to a whole group of 4, reading a valid code: that
            // of node 2 lane (one bank per lane) with two or more nodes per
            // lane, the lane's own node with one
            const uint32_t pad = codes + (npl == 1 ? 2u : 4u) * (uint32_t)lane;
            for (int d = net.D[k]; d < groups4(net.D[k]); ++d)
                lut[(o + d) * 32 + lane] = 0x04040000u | (pad & 0xffffu);
            o += groups4(net.D[k]);
            const int i = net.q_node[lane * npl + k];
            uint32_t u = 1, m1 = 1, d2 = 0;
            if (i >= 0) {
                u = net.sync ? 0u : (uint32_t)x[3 * E + i];
                m1 = (uint32_t)x[3 * E + N + i] + 1u;
                d2 = x[3 * E + 2 * N + i] == 2 ? 0xffffffffu : 0u;
            }
            F(k, kF_U2, lane) = u * 0x00010001u;
            F(k, kF_CM, lane) = (128u - m1) * kB1;
            F(k, kF_D2, lane) = d2;
        }
    }

    // Candidate change of edge idx (its table entry is owned by lane `owner`).
    __device__ void change_edge(const DevNet &net, int lane, int owner, int pos, int w, int p,
                                int t, int /*idx*/)
    {
        if (lane != owner) return;
        const int row = lut_row(net, (pos >> 8) & 0xff, pos & 0xff);
        const uint32_t a = (uint32_t)(row * 32 + lane);
        const uint32_t old = lut[a];
        undo_lut = true;
        undo_addr = a;
        undo_val = old;
        lut[a] = edge_word_s(w, p, t, old);
    }

    // Candidate change of node parameter (kind 3: u, 4: m, 5: d) of slot k.
    __device__ void change_node(int lane, int owner, int k, int kind, int v)
    {
        if (lane != owner) return;
        const int f = kind == 3 ? kF_U2 : kind == 4 ? kF_CM : kF_D2;
        const uint32_t a = (uint32_t)((k * kF_N + f) * 32 + lane);
        undo_lut = false;
        undo_addr = a;
        undo_val = node[a];
        node[a] = kind == 3 ? (uint32_t)v * 0x00010001u
                : kind == 4 ? (127u - (uint32_t)v) * kB1
                            : (v == 2 ? 0xffffffffu : 0u);
    }

    __device__ void undo(int lane, int owner)
    {
        if (lane != owner) return;
        if (undo_lut) lut[undo_addr] = undo_val;
        else node[undo_addr] = undo_val;
    }

    // 16-bit code of a node: nibble c = 4 - s_c.
    __device__ __forceinline__ static uint16_t code_of(uint32_t s4)
    {
        const uint32_t v = 4u * kB1 - s4;
        const uint32_t x = v | (v >> 4);
        return (uint16_t)prmt(x, 0u, 0x4420u);
    }

    // Simulate(x) of Table 1 (Sections 2.1-2.3), 4 conditions per group, the
    // byte-SIMD update of simulate_swar4 with its state in shared memory.
    __device__ int32_t simulate(const DevNet &net, int lane, uint8_t *traj,
                                int32_t limit = INT32_MAX)
    {
        // the early-rejection check lives only in the instance that needs it
        return limit == INT32_MAX ? simulate_t<false>(net, lane, traj, limit)
                                  : simulate_t<true>(net, lane, traj, limit);
    }

    template <bool EARLY>
    __device__ __forceinline__ int32_t simulate_t(const DevNet &net, int lane, uint8_t *traj,
                                                  int32_t limit)
    {
        const int T = net.T;
        uint16_t *code = reinterpret_cast<uint16_t *>(sm + codes);
        uint32_t score = 0;
        for (int g = 0; g < net.G; ++g) {
            for (int k = 0; k < npl; ++k) {
                const size_t q = (size_t)g * 32 * npl + lane * npl + k;
                const uint32_t s4 = __ldg(net.init_s4 + q);
                F(k, kF_S4, lane) = s4;
                F(k, kF_CU, lane) = 0;
                F(k, kF_CD, lane) = 0;
                F(k, kF_UA01, lane) = F(k, kF_U2, lane);
                F(k, kF_UA23, lane) = F(k, kF_U2, lane);
                F(k, kF_MOV, lane) = __ldg(net.movable + q);
                code[lane * npl + k] = code_of(s4);
            }
            const int ncg = min(net.C - 4 * g, 4);
            for (int tau = 0; tau < T; ++tau) {
                if (tau > 0) {
                    if (net.async) {   // only the step's selected node may move
                        const uint32_t *mt = net.movable_t + ((size_t)(g * T + tau) * 32 + lane) * npl;
                        for (int k = 0; k < npl; ++k) F(k, kF_MOV, lane) = __ldg(mt + k);
                    }
                    uint32_t m01 = 0, m23 = 0;
                    int o = 0;
                    for (int k = 0; k < npl; ++k) {
                        const int D4 = groups4(net.D[k]);
                        const uint32_t acc = gather_rows<32>(lut + o * 32 + lane, D4, sm);
                        o += D4;
                        const uint32_t s4 = F(k, kF_S4, lane);
                        const uint32_t tgt = target4(acc);
                        const uint32_t dp = tgt + 2 * kB1 - s4;
                        const uint32_t up = (dp + 0x7D7D7D7Du) & kH;
                        const uint32_t dn = ~(dp + 0x7E7E7E7Eu) & kH;
                        const uint32_t cu = (F(k, kF_CU, lane) + kB1) & prmt(up, 0u, 0xBA98u);
                        const uint32_t cd = (F(k, kF_CD, lane) + kB1) & prmt(dn, 0u, 0xBA98u);
                        F(k, kF_CU, lane) = cu;
                        F(k, kF_CD, lane) = cd;
                        const uint32_t cm = F(k, kF_CM, lane);
                        const uint32_t el = ((cu + cm) | (cd + cm)) & F(k, kF_MOV, lane);
                        const uint32_t d2 = F(k, kF_D2, lane);
                        const uint32_t step1 = s4 + (up >> 7) - (dn >> 7);
                        F(k, kF_SN, lane) = (tgt & d2) | (step1 & ~d2);
                        F(k, kF_ELM, lane) = prmt(el, 0u, 0xBA98u);
                        const uint32_t p01 = F(k, kF_UA01, lane) & prmt(el, 0u, 0x9988u);
                        const uint32_t p23 = F(k, kF_UA23, lane) & prmt(el, 0u, 0xBBAAu);
                        F(k, kF_PR01, lane) = p01;
                        F(k, kF_PR23, lane) = p23;
                        m01 = max_u16x2(m01, p01);
                        m23 = max_u16x2(m23, p23);
                    }
                    const uint32_t p0 = __reduce_max_sync(kFull, m01 & 0xffffu);
                    const uint32_t p1 = __reduce_max_sync(kFull, m01 >> 16);
                    const uint32_t p2 = __reduce_max_sync(kFull, m23 & 0xffffu);
                    const uint32_t p3 = __reduce_max_sync(kFull, m23 >> 16);
                    const uint32_t P01 = prmt(p0, p1, 0x5410u), P23 = prmt(p2, p3, 0x5410u);
                    for (int k = 0; k < npl; ++k) {
                        const uint32_t nz01 =
                            ((F(k, kF_PR01, lane) ^ P01) + 0x7FFF7FFFu) & 0x80008000u;
                        const uint32_t nz23 =
                            ((F(k, kF_PR23, lane) ^ P23) + 0x7FFF7FFFu) & 0x80008000u;
                        const uint32_t upd = F(k, kF_ELM, lane) & ~prmt(nz01, nz23, 0xFDB9u);
                        const uint32_t s4 = (F(k, kF_S4, lane) & ~upd) | (F(k, kF_SN, lane) & upd);
                        F(k, kF_S4, lane) = s4;
                        F(k, kF_CU, lane) &= ~upd;
                        F(k, kF_CD, lane) &= ~upd;
                        const uint32_t u2 = F(k, kF_U2, lane);
                        const uint32_t u01 = prmt(upd, 0u, 0x9988u), u23 = prmt(upd, 0u, 0xBBAAu);
                        F(k, kF_UA01, lane) = ((F(k, kF_UA01, lane) + u2) & ~u01) | (u2 & u01);
                        F(k, kF_UA23, lane) = ((F(k, kF_UA23, lane) + u2) & ~u23) | (u2 & u23);
                        code[lane * npl + k] = code_of(s4);
                    }
                }
                __syncwarp();
                // error at this time point (compact entry words)
                const uint32_t *ob = net.obs + (((size_t)g * T + tau) * 32 + lane) * npl;
                for (int k = 0; k < npl; ++k) {
                    const uint32_t s4 = F(k, kF_S4, lane);
                    score = entry_error(s4, __ldg(ob + k), score);
                    if (traj) {
                        const int i = net.q_node[lane * npl + k];
                        for (int c = 0; c < ncg; ++c)
                            if (i >= 0)
                                traj[((size_t)(4 * g + c) * T + tau) * net.N + i] =
                                    (uint8_t)((s4 >> (8 * c)) & 0xffu);
                    }
                }
                if (EARLY && (tau & 3) == 3) {
                    // exact early rejection: the partial score never decreases
                    const uint32_t tot = __reduce_add_sync(kFull, score) >> 2;
                    if (tot > (uint32_t)limit) return (int32_t)tot;
                }
            }
            __syncwarp();
        }
        return (int32_t)(__reduce_add_sync(kFull, score) >> 2);   // quarter units
    }
};

// Hybrid path for 6 or 8 nodes per lane (129 .. 256 nodes): the table words of
// the shared-memory path (16-bit code address, code nibble 4 - s) stay in the
// warp's shared memory, gathered in groups of 4 rows, while the per-node
// byte-SIMD update state lives in registers (the simulation of rn_device.cuh,
// simulate_swar4_core), so that only the gather touches shared memory.
constexpr int kSmemRegSlots[3] = {6, 8, 10};
// Blocks of 4 warps per SM the hybrid kernels are compiled for: 3 (at most
// 168 registers a thread) up to 8 nodes per lane; 10 nodes per lane keep their
// node state in up to 255 registers at 2 blocks.
template <int NPL>
constexpr int smemreg_min_blocks()
{
    return NPL > 8 ? 2 : 3;
}

__host__ __device__ inline uint32_t smem_reg_warp_bytes(uint32_t lut_words, int pstride, int N)
{
    const uint32_t cnt = 2u * (((uint32_t)N + 15u) & ~15u);
    return lut_words * 4u + (uint32_t)pstride + cnt;
}

template <int NPL>
struct SmemRegPath {
    uint8_t *sm;         // dynamic shared memory of the block
    uint32_t codes;      // offset of this warp's code array in sm
    uint32_t *lut;       // [sum groups4(D_k)][32]
    int32_t u[NPL], m1[NPL], d2[NPL];
    uint32_t undo_addr, undo_val;
    int undo_kind, undo_slot;

    __device__ __forceinline__ int lut_row(const DevNet &net, int k, int d) const
    {
        int o = 0;
        for (int kk = 0; kk < k; ++kk) o += groups4(net.D[kk]);
        return o + d;
    }

    __device__ void load(const DevNet &net, const int8_t *x, int lane)
    {
        const int E = net.E, N = net.N;
        const uint32_t pad = codes + 4u * (uint32_t)lane;   // the code of node 2 lane
        int o = 0;
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
            for (int d = 0; d < net.D[k]; ++d) {
                const int e = net.edge_id[(k * net.dtab + d) * 32 + lane];
                uint32_t w;
                if (e >= 0)
                    w = edge_word_s(x[e], x[E + e], x[2 * E + e],
                                    codes + 2u * (uint32_t)net.node_q[net.src[e]]);
                else
                    w = 0x04040000u | ((codes + (uint32_t)(-1 - e)) & 0xffffu);
                lut[(o + d) * 32 + lane] = w;
            }
            for (int d = net.D[k]; d < groups4(net.D[k]); ++d)
                lut[(o + d) * 32 + lane] = 0x04040000u | (pad & 0xffffu);
            o += groups4(net.D[k]);
            const int i = net.q_node[lane * NPL + k];
            u[k] = i >= 0 ? (net.sync ? 0 : x[3 * E + i]) : 1;
            m1[k] = i >= 0 ? x[3 * E + N + i] + 1 : 1;
            d2[k] = i >= 0 ? x[3 * E + 2 * N + i] == 2 : 0;
        }
    }

    __device__ void change_edge(const DevNet &net, int lane, int owner, int pos, int w, int p,
                                int t, int)
    {
        if (lane != owner) return;
        const uint32_t a = (uint32_t)(lut_row(net, (pos >> 8) & 0xff, pos & 0xff) * 32 + lane);
        undo_kind = 0;
        undo_addr = a;
        undo_val = lut[a];
        lut[a] = edge_word_s(w, p, t, undo_val);
    }

    __device__ void change_node(int lane, int owner, int slot, int kind, int v)
    {
        if (lane != owner) return;
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

    __device__ void undo(int lane, int owner)
    {
        if (lane != owner) return;
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

    __device__ int32_t simulate(const DevNet &net, int lane, uint8_t *traj,
                                int32_t limit = INT32_MAX)
    {
        SlotGather<NPL, 32, (NPL > 6)> gather;
        gather.lut = lut + lane;
        gather.sm = sm;
        int o = 0;
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
            gather.row0[k] = o;
            gather.d4[k] = groups4(net.D[k]);
            o += gather.d4[k];
        }
        if (limit == INT32_MAX)
            return simulate_swar4_core<NPL, true, false>(u, m1, d2, net, sm, codes, lane, traj,
                                                         limit, gather);
        return simulate_swar4_core<NPL, true, true>(u, m1, d2, net, sm, codes, lane, traj, limit,
                                                    gather);
    }
};

}  // namespace rn
