// rn_device.cuh -- device-side data layout and the warp-per-chain simulator.
//
// One warp owns one parameter vector (one annealing chain).  Node i of the
// network lives in lane l, slot k (internal index q = l * NPL + k); nodes are
// ranked by in-degree so that the 32 nodes of a slot have similar in-degree,
// and every slot k is padded to one in-degree D_k across the warp.
//
// Conditions are simulated CG at a time (CG = 1, 2 or 4).  The warp's node
// states live in shared memory as one 16-bit code per node whose nibble c is
// the state of condition c of the group: the gather source of the image.
//
// Each lane keeps, in registers, one 32-bit table word per in-edge of its nodes:
//
//   byte b (b = 0, 1, 2) = 4 + (b // t) * w * p     image term of a source in state b
//   byte 3               = 2 * q_src                shared-memory offset of the source code
//
// (Section 2.1).  PRMT (__byte_perm) of the table word with the 16-bit code of
// the source as selector places the biased image term of condition c in byte
// c, so one shared load, two PRMTs and one add give the image terms of CG
// conditions at once; after D_k edges byte c holds 4 D_k + K_i (<= 128 for
// D_k <= 16, so no byte carries into the next).  The priority maximum of
// Section 2.2 is one redux.sync per condition.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rn {

constexpr int kMaxSlots = 16;         // nodes per lane (N <= 512)
constexpr int kRegSlots = 4;          // nodes per lane of the register-table kernels (N <= 128)
constexpr uint32_t kFull = 0xffffffffu;
constexpr int32_t kOutUA = -(1 << 22);   // priority seed of a node that never moves

// Network as the kernels see it (all pointers are device memory).
constexpr int kBlockLanes = 256;        // threads of a chain on the block path (N > 512)

struct DevNet {
    int32_t N, E, P, n_free;
    int32_t C, T, G;                    // conditions, time points, condition groups
    int32_t npl, cg, dtab;              // nodes per lane, conditions per group, table stride
    int32_t lanes;                      // threads per chain: 32 (a warp) or kBlockLanes
    int32_t sync;                       // 1: every eligible node has the same priority
                                        //    (synchronous and asynchronous schemes)
    int32_t async;                      // 1: asynchronous scheme, movable_t below
    int32_t D[kMaxSlots];               // padded in-degree of each slot
    const int32_t *edge_id;             // [npl][dtab][32] edge index, or -1 - (code offset) for padding
    const uint8_t *warp_d4;             // [npl][lanes / 32] rows of each slot a warp gathers
                                        // (block path; null on the warp paths)
    const uint8_t *edge_q2;             // [E] 2 * internal index of the edge's source
    const int32_t *edge_pos;            // [E] (lane << 16) | (slot << 8) | d
    const int32_t *node_q;              // [N] internal index of node i
    const int16_t *q_node;              // [32 * npl] node at internal index q, or -1
    const int32_t *src, *dst;           // [E]
    const uint8_t *fast;                // [N]
    const int32_t *free_list;           // [n_free] free parameter indices, ascending
    const int32_t *in_ptr, *in_edges;   // in-edges of each node, ascending edge index
    const int32_t *out_ptr, *out_edges; // out-edges of each node, ascending edge index
    const uint8_t *frozen;              // [P] or null
    const int8_t *frozen_val;           // [P] or null
    const uint16_t *init_code;          // [G][32 * npl] initial state codes of a group
    const uint16_t *out_bits;           // [G][32] bit (k * cg + c): never moves
    const uint32_t *init_s4;            // [G][32 * npl] byte c: initial state, condition c
    const uint32_t *movable;            // [G][32 * npl] bit 7 of byte c: may move in c
    const uint32_t *movable_t;          // [G][T][lanes * npl] the same per step under the
                                        // asynchronous scheme (only the selected node)
    const int32_t *async_sel;           // [C][T] the selected node of each step (scalar path)
    const uint32_t *obs;                // [C][T][32][npl] error table of each entry
};

// Chain state of one network.
struct DevChains {
    int32_t n;
    int32_t pstride;                    // bytes per chain row (P rounded up to 16)
    uint64_t seed;
    int8_t *x_cur, *x_best;             // [n][pstride]
    int32_t *d_cur, *d_best;            // [n]
    int64_t *cnt;                       // [n][3] accepted, accepted uphill, null
};

// Steps [g0, g1) of one launch and the acceptance tables of their levels.
// The steps of every chain are cut into chunks of `chunk` steps; the work
// items (chunk j, chain c) are handed out in order j * n + c from a queue, and
// item (j, c) starts once chunk j - 1 of chain c is done.
struct DevSched {
    int64_t g0, g1;
    int64_t iters;                      // proposals per level
    int64_t level0;                     // level of thr_off[0]
    int32_t reset_to_best;
    int32_t early_reject;               // stop simulating candidates that cannot be accepted
    int64_t chunk;                      // steps per work item
    int32_t n_chunks;
    const int32_t *thr_off;             // [levels] start of the level's table
    const int32_t *thr_len;             // [levels] D_l: largest dE with a nonzero threshold
    const uint32_t *thr;                // entries for dE = 1 .. D_l
    unsigned int *queue;                // next work item (zeroed before the launch)
    int32_t *done;                      // [n] chunks finished per chain (zeroed before the launch)
    int32_t *err;                       // set to 1 when a wait gives up
};

constexpr int kWaitLimit = 1 << 22;     // polls of a predecessor flag before giving up

// GetCandidate's new value (Table 1): the pick(r1)-th, in ascending order, of
// the values of a kind-`kind` parameter's domain other than cur and, where
// blocked0, other than 0 (the constraints of Section 2.5.3); false when none is
// left (blocked_all, or nothing besides cur).  Every domain is a run of
// consecutive integers (Section 2.1: w 0..2, p -1..1, t 1..2; Section 2.2: u
// 1..6, or 10..12 for a fast node, m 0..2, d 1..2), so the value is the run's
// pick-th with the excluded values stepped over, in ascending order, which
// needs no per-kind branch (lanes of a warp that hold different kinds do not
// diverge).  blocked0 arises only for w != 0, whose run starts at 0.
__host__ __device__ __forceinline__ bool pick_alternative(int kind, bool fast, int cur,
                                                          bool blocked0, bool blocked_all,
                                                          uint32_t r1, int &v)
{
    // per kind, in nibble k: the run's lowest value + 1, and its length
    int lo = (int)((0x212201u >> (4 * kind)) & 15u) - 1;
    int n = (int)((0x236233u >> (4 * kind)) & 15u);
    if (fast && kind == 3) {
        lo = 10;
        n = 3;
    }
    const int n_alt = blocked_all ? 0 : n - 1 - (blocked0 ? 1 : 0);
    if (n_alt <= 0) return false;
#ifdef __CUDA_ARCH__
    const uint32_t m = __umulhi(r1, (uint32_t)n_alt);
#else
    const uint32_t m = (uint32_t)(((uint64_t)r1 * (uint32_t)n_alt) >> 32);
#endif
    v = lo + (int)m;
    if (blocked0 && v >= 0) ++v;
    if (v >= cur) ++v;
    return true;
}

// Block and index of parameter j in x = [w(E), p(E), t(E), u(N), m(N), d(N)]
// (Section 2.5): kind 0..5 and the index within its block, by comparisons
// (a division by the run-time E or N is a long dependent sequence on the
// proposal's path).
__host__ __device__ __forceinline__ void param_kind(int j, int E, int N, int &kind, int &idx)
{
    if (j < 3 * E) {
        kind = (j >= E) + (j >= 2 * E);
        idx = j - kind * E;
    } else {
        const int t = j - 3 * E;
        const int k = (t >= N) + (t >= 2 * N);
        kind = 3 + k;
        idx = t - k * N;
    }
}

// The block path's register variant (2, 4, 6 or 8 nodes per thread) keeps two
// copies of the chain's 16-bit state codes in shared memory.  Word w of the
// first copy (codes of internal indices 2w and 2w + 1) is word code_word2(w) of
// the second: each row of 32 words (one word per bank) rotated by its row
// index, so that codes that share a bank in the first copy sit in different
// banks of the second.  The host's layout picks, for every table entry, the
// copy that keeps the 32 lanes of a warp on distinct banks in that row; an
// entry of edge_id with kCodeCopy2 set reads the second copy.  (A network
// whose tables leave no room for the second copy keeps one.)
constexpr int32_t kCodeCopy2 = 1 << 30;
__host__ __device__ __forceinline__ bool block_reg_npl(int npl)
{
    return npl == 2 || npl == 4 || npl == 6 || npl == 8;
}
__host__ __device__ __forceinline__ uint32_t code_word2(uint32_t w)
{
    return (w & ~31u) | ((w + (w >> 5)) & 31u);
}
// Shared memory one block may use (227 KiB on sm_103).
constexpr uint32_t kBlockSmemMax = 232448u;
// Bytes of one copy of the block path's codes (kBlockLanes x npl), rounded to 256.
__host__ __device__ __forceinline__ uint32_t block_code_bytes(int npl)
{
    return (2u * (uint32_t)kBlockLanes * (uint32_t)npl + 255u) & ~255u;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; each round
// multiplies counter words 0 and 2 by 0xD2511F53 / 0xCD9E8D57 and crosses the
// high halves with words 1 and 3 and the key; the key is bumped by the Weyl
// constants 0x9E3779B9 / 0xBB67AE85 between rounds.
__device__ __forceinline__ uint4 philox(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                                        uint32_t c3)
{
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a = 0xD2511F53u * c0, ah = __umulhi(0xD2511F53u, c0);
        const uint32_t b = 0xCD9E8D57u * c2, bh = __umulhi(0xCD9E8D57u, c2);
        c0 = bh ^ c1 ^ k0;
        c1 = b;
        c2 = ah ^ c3 ^ k1;
        c3 = a;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

// floor(r * n / 2^32): uniform index in [0, n).
__device__ __forceinline__ uint32_t pick(uint32_t r, uint32_t n) { return __umulhi(r, n); }

// Table word of an edge (Section 2.1): byte b = 4 + (b // t) * w * p, byte 3 = q2.
__host__ __device__ __forceinline__ uint32_t edge_word(int w, int p, int t, uint32_t q2)
{
    const int wp = w * p;
    const int f1 = (t == 1) ? wp : 0;
    const int f2 = (t == 1) ? 2 * wp : wp;
    return 0x04u | ((uint32_t)(4 + f1) << 8) | ((uint32_t)(4 + f2) << 16) | (q2 << 24);
}

// Per-lane register copy of a chain's parameters: slot 0 holds up to D0
// in-edges, slots 1 .. NPL-1 up to D1.
template <int NPL, int D0, int D1>
struct Regs {
    uint32_t lut0[D0];
    uint32_t lutr[NPL > 1 ? NPL - 1 : 1][D1];
    int32_t u[NPL];            // speed
    int32_t m1[NPL];           // memory + 1
    int32_t d2[NPL];           // 1 if step size 2
};

// Visit the table word of (slot k, edge d) with compile-time k and d.
template <int NPL, int D0, int D1, typename F>
__device__ __forceinline__ void for_each_word(Regs<NPL, D0, D1> &R, F f)
{
#pragma unroll
    for (int d = 0; d < D0; ++d) f(0, d, R.lut0[d]);
#pragma unroll
    for (int k = 1; k < NPL; ++k)
#pragma unroll
        for (int d = 0; d < D1; ++d) f(k, d, R.lutr[k - 1][d]);
}

// Fill a lane's registers from a parameter vector x (any address space).
template <int NPL, int D0, int D1>
__device__ __forceinline__ void load_regs(Regs<NPL, D0, D1> &R, const DevNet &net, const int8_t *x,
                                          int lane)
{
    const int E = net.E, N = net.N;
    for_each_word<NPL, D0, D1>(R, [&](int k, int d, uint32_t &word) {
        // padding: f = 0, reading a valid state code (its nibbles select one of
        // the three 4s): that of node 2 lane (one bank per lane) with two or
        // more nodes per lane, the lane's own node with one
        uint32_t w = 0x00040404u | ((uint32_t)((NPL == 1 ? 2 : 4) * lane) << 24);
        if (d < net.D[k]) {
            const int e = net.edge_id[(k * net.dtab + d) * 32 + lane];
            if (e >= 0) w = edge_word(x[e], x[E + e], x[2 * E + e], net.edge_q2[e]);
            else w = 0x00040404u | ((uint32_t)(-1 - e) << 24);   // padding reading a shared word
        }
        word = w;
    });
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
        const int i = net.q_node[lane * NPL + k];
        if (i >= 0) {
            R.u[k] = net.sync ? 0 : x[3 * E + i];   // synchronous: every priority 0
            R.m1[k] = x[3 * E + N + i] + 1;
            R.d2[k] = x[3 * E + 2 * N + i] == 2;
        } else {
            R.u[k] = 1;
            R.m1[k] = 1;
            R.d2[k] = 0;
        }
    }
}

// Edges per slot rounded up to whole groups of 4; the table words past D are
// neutral (every byte 4), so a group-of-4 gather adds exactly 4 per padding
// word and condition.
__host__ __device__ __forceinline__ int groups4(int D) { return (D + 3) & ~3; }

// Biased image terms of the slot's node for the CG conditions, one byte each:
// `acc` plus the sum over its first groups4(D) table words (4 per padding
// word).  Edges go in groups of 4, the four shared-memory loads of a group
// issued before their uses; D is warp uniform, so the groups do not diverge.
template <int DC>
__device__ __forceinline__ uint32_t image(const uint32_t (&lut)[DC], int D, uint32_t base,
                                          const uint8_t *sm, uint32_t acc = 0)
{
    static_assert(DC % 4 == 0, "table capacities are multiples of 4");
#pragma unroll
    for (int g = 0; g < DC; g += 4) {
        if (g < D) {
            uint32_t c[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                c[i] = *(const uint16_t *)(sm + __byte_perm(lut[g + i], base, 0x7653u));
#pragma unroll
            for (int i = 0; i < 4; ++i) acc += __byte_perm(lut[g + i], 0u, c[i]);
        }
    }
    return acc;
}

template <int NPL, int D0, int D1>
__device__ __forceinline__ void images(uint32_t (&acc)[NPL], const Regs<NPL, D0, D1> &R,
                                       const DevNet &net, uint32_t base, const uint8_t *sm)
{
    acc[0] = image<D0>(R.lut0, net.D[0], base, sm);
    if constexpr (NPL > 1) {
#pragma unroll
        for (int k = 1; k < NPL; ++k) acc[k] = image<D1>(R.lutr[k - 1], net.D[k], base, sm);
    }
}

// Byte-SIMD helpers: prmt with sign replication (selector nibble bit 3 set
// copies the top bit of the selected byte into all 8 bits of the result byte),
// and the 16-bit-lane maximum.
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

__device__ __forceinline__ uint32_t max_u16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

constexpr uint32_t kB1 = 0x01010101u;   // 1 in every byte
constexpr uint32_t kH = 0x80808080u;    // top bit of every byte

// Biased image bytes: a gather starts every byte at kImage0 - 4 D4 and adds
// 4 + f per table word, so a byte ends at 127 + K_i (in 63 .. 191 for D <= 16,
// and the block path's larger in-degrees stay inside the byte too).  Then bit
// 7 of a byte is [K >= 1] and bit 7 of the byte minus 1 is [K >= 2], and their
// sum is clamp(K, 0, 2), the target of Section 2.2 (reading 3).
constexpr uint32_t kImage0 = kH - kB1;

__device__ __forceinline__ uint32_t target4(uint32_t a)
{
    return ((a >> 7) & kB1) + (((a - kB1) >> 7) & kB1);
}

// One group of four table rows (words w, state codes read through their
// address halves) added into acc; the next group's words are loaded into wn
// first when there is one (rows d + 4 .. d + 7 of D4).
template <int STRIDE>
__device__ __forceinline__ void gather_group(const uint32_t (&w)[4], uint32_t (&wn)[4],
                                             const uint32_t *lw, int d, int D4,
                                             const uint8_t *sm, uint32_t &acc)
{
    uint32_t c[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) c[i] = *reinterpret_cast<const uint16_t *>(sm + (w[i] & 0xffffu));
    if (d + 4 < D4) {
#pragma unroll
        for (int i = 0; i < 4; ++i) wn[i] = lw[(d + 4 + i) * STRIDE];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) acc += prmt(w[i], 0x04040404u, c[i]);
}

// Biased image bytes of one slot from its D4 = groups4(D) shared-memory table
// rows at lw (row stride STRIDE words; word = code address | prmt selectors):
// kH - 4 D4 per byte plus, per row, the source's state code picked into the
// byte of each condition.  With PIPE the next group's four words are loaded
// before the current group's codes are used, so that two groups are in flight
// (measured faster with 8 nodes per lane, slower with 6); the loop alternates
// between two word buffers, so nothing is copied from one to the other.
template <int STRIDE, bool PIPE = true>
__device__ __forceinline__ uint32_t gather_rows(const uint32_t *lw, int D4, const uint8_t *sm)
{
    uint32_t acc = kImage0 - 0x04040404u * (uint32_t)D4;
    if constexpr (!PIPE) {
        for (int d = 0; d < D4; d += 4) {
            uint32_t w[4], c[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) w[i] = lw[(d + i) * STRIDE];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                c[i] = *reinterpret_cast<const uint16_t *>(sm + (w[i] & 0xffffu));
#pragma unroll
            for (int i = 0; i < 4; ++i) acc += prmt(w[i], 0x04040404u, c[i]);
        }
        return acc;
    }
    if (D4 == 0) return acc;
    // w1 is read only after the group before has loaded it
    uint32_t w0[4], w1[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) w0[i] = lw[i * STRIDE];
    for (int d = 0;;) {
        gather_group<STRIDE>(w0, w1, lw, d, D4, sm, acc);
        if ((d += 4) >= D4) break;
        gather_group<STRIDE>(w1, w0, lw, d, D4, sm, acc);
        if ((d += 4) >= D4) break;
    }
    return acc;
}

// Two slots' images at once (slots of equal row counts, laid out one after the
// other): the same loop as gather_rows over both, so that twice the table words
// and state codes are in flight.
template <int STRIDE>
__device__ __forceinline__ void gather_rows_pair(const uint32_t *la, const uint32_t *lb, int D4,
                                                 const uint8_t *sm, uint32_t &acc_a,
                                                 uint32_t &acc_b)
{
    acc_a = kImage0 - 0x04040404u * (uint32_t)D4;
    acc_b = acc_a;
    if (D4 == 0) return;
    // a1 and b1 are read only after the group before has loaded them
    uint32_t a0[4], b0[4], a1[4], b1[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        a0[i] = la[i * STRIDE];
        b0[i] = lb[i * STRIDE];
    }
    for (int d = 0;;) {
        gather_group<STRIDE>(a0, a1, la, d, D4, sm, acc_a);
        gather_group<STRIDE>(b0, b1, lb, d, D4, sm, acc_b);
        if ((d += 4) >= D4) break;
        gather_group<STRIDE>(a1, a0, la, d, D4, sm, acc_a);
        gather_group<STRIDE>(b1, b0, lb, d, D4, sm, acc_b);
        if ((d += 4) >= D4) break;
    }
}

// A gather functor that also serves two slots at once (pair(k, a, b) for slots
// k and k + 1) advertises it with kPair; simulate_swar4_core then gathers in
// pairs.
template <class G, class = void>
struct gathers_pairs {
    static constexpr bool value = false;
};
template <class G>
struct gathers_pairs<G, decltype((void)G::kPair)> {
    static constexpr bool value = G::kPair;
};

// The image gather of the shared-memory table layouts (hybrid and block
// paths): slot k's rows start at row0[k] of this thread's column and number
// d4[k]; slots 2j and 2j + 1 have equal row counts (the layout pads them so),
// so they are gathered in pairs.
template <int NPL, int STRIDE, bool PIPE>
struct SlotGather {
    static constexpr bool kPair = true;
    const uint32_t *lut;   // this thread's column of the table rows
    const uint8_t *sm;
    int row0[NPL], d4[NPL];
    __device__ __forceinline__ uint32_t operator()(int k) const
    {
        return gather_rows<STRIDE, PIPE>(lut + row0[k] * STRIDE, d4[k], sm);
    }
    __device__ __forceinline__ void pair(int k, uint32_t &a, uint32_t &b) const
    {
        gather_rows_pair<STRIDE>(lut + row0[k] * STRIDE, lut + row0[k + 1] * STRIDE, d4[k], sm,
                                 a, b);
    }
};

template <int NPL>
__device__ __forceinline__ void store_codes(uint8_t *p, const uint32_t (&code)[NPL])
{
    if constexpr (NPL == 1) {
        *reinterpret_cast<uint16_t *>(p) = (uint16_t)code[0];
    } else if constexpr (NPL == 2) {
        *reinterpret_cast<uint32_t *>(p) = code[0] | (code[1] << 16);
    } else if constexpr (NPL == 4) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(code[0] | (code[1] << 16),
                                                   code[2] | (code[3] << 16));
    } else if constexpr (NPL == 8) {
        *reinterpret_cast<uint4 *>(p) =
            make_uint4(code[0] | (code[1] << 16), code[2] | (code[3] << 16),
                       code[4] | (code[5] << 16), code[6] | (code[7] << 16));
    } else {
        static_assert(NPL % 2 == 0, "codes are stored in pairs");
#pragma unroll
        for (int k = 0; k < NPL; k += 2)
            reinterpret_cast<uint32_t *>(p)[k / 2] = code[k] | (code[k + 1] << 16);
    }
}

template <int NPL>
__device__ __forceinline__ void load_codes(uint32_t (&code)[NPL], const uint16_t *p)
{
    if constexpr (NPL == 1) {
        code[0] = p[0];
    } else if constexpr (NPL == 2) {
        const uint32_t v = *reinterpret_cast<const uint32_t *>(p);
        code[0] = v & 0xffffu; code[1] = v >> 16;
    } else {
        const uint2 v = *reinterpret_cast<const uint2 *>(p);
        code[0] = v.x & 0xffffu; code[1] = v.x >> 16;
        code[2] = v.y & 0xffffu; code[3] = v.y >> 16;
    }
}

template <int NPL>
__device__ __forceinline__ void load_obs(uint32_t (&w)[NPL], const uint32_t *ob)
{
    if constexpr (NPL % 4 == 0) {
#pragma unroll
        for (int k = 0; k < NPL; k += 4) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(ob + k));
            w[k] = v.x; w[k + 1] = v.y; w[k + 2] = v.z; w[k + 3] = v.w;
        }
    } else if constexpr (NPL % 2 == 0) {
#pragma unroll
        for (int k = 0; k < NPL; k += 2) {
            const uint2 v = __ldg(reinterpret_cast<const uint2 *>(ob + k));
            w[k] = v.x; w[k + 1] = v.y;
        }
    } else if constexpr (NPL == 2) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(ob));
        w[0] = v.x; w[1] = v.y;
    } else {
        w[0] = __ldg(ob);
    }
}

// Simulate(x) for groups of 4 conditions, with the priority update of
// Section 2.2 done byte-SIMD within registers: byte c of every per-node word
// belongs to condition c of the group.
//
//   a    = image byte 127 + K_i (the accumulator starts at kImage0 - 4 D4 per byte)
//   tgt  = [K >= 1] + [K >= 2] = clamp(K, 0, 2)      (bit 7 of a and of a - 1)
//   dp   = tgt - s + 2 in [0, 4]; UP = dp >= 3, DN = dp <= 1 (told to move up/down)
//   cu   = consecutive up drives, cd = consecutive down drives (reset by a move)
//   EL   = cu >= m + 1 or cd >= m + 1, only where the node may move
//   ua   = u * (steps since the last update), 16-bit lanes (two words)
//   the nodes whose eligible priority equals the warp maximum of their
//   condition move to tgt (d = 2) or one level toward it (d = 1).
// Byte values stay within their byte: a in [3, 251] for D <= 31, counters
// below 128 for T <= 128, priorities below 2^15.
// 16-bit state code of a node's four conditions: nibble c = s_c for the
// register-table words, 4 - s_c for the shared-memory words (rn_smem.cuh).
template <bool SMEM_FMT>
__device__ __forceinline__ uint32_t state_code(uint32_t s4)
{
    const uint32_t v = SMEM_FMT ? 4u * kB1 - s4 : s4;
    return prmt(v | (v >> 4), 0u, 0x4420u);
}

// The state codes of two nodes in one word (the first in the low half), as
// the shared-memory code array holds them: one byte permutation for the pair.
template <bool SMEM_FMT>
__device__ __forceinline__ uint32_t state_code_pair(uint32_t s4a, uint32_t s4b)
{
    const uint32_t va = SMEM_FMT ? 4u * kB1 - s4a : s4a;
    const uint32_t vb = SMEM_FMT ? 4u * kB1 - s4b : s4b;
    return prmt(va | (va >> 4), vb | (vb >> 4), 0x6420u);
}

// Store the state codes of a thread's NPL nodes (2 bytes each, node k at p + 2 k).
template <int NPL, bool SMEM_FMT>
__device__ __forceinline__ void store_state_codes(uint8_t *p, const uint32_t (&s4)[NPL])
{
    if constexpr (NPL == 1) {
        *reinterpret_cast<uint16_t *>(p) = (uint16_t)state_code<SMEM_FMT>(s4[0]);
    } else {
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
    }
}

// Error of a node's four conditions at one time point (Section 2.3) from its
// compact entry word (byte c = R_c | W_c << 2, W = 0 where unobserved), added
// to acc in quarter units: 4 sum_c W_c |s_c - R_c|.  For s, R in 0..2, x = s ^ R
// equals |s - R| except x = 3 (s, R = 1, 2), where |s - R| = 1 = x - 2; DP4A
// weights the four bytes by 4 W (the word's bits 2-3 in place) and sums them.
// Scores are below 2^30 (checked when the time course is loaded), so the
// quarter-unit sums fit 32 bits; y = sum >> 2.
__device__ __forceinline__ uint32_t entry_error(uint32_t s4, uint32_t word, uint32_t acc)
{
    const uint32_t x = s4 ^ (word & 0x03030303u);
    const uint32_t d = x - ((x & (x >> 1) & kB1) << 1);
    return __dp4a(d, word & 0x0c0c0c0cu, acc);
}

// Reductions and barriers of a chain simulated by one warp (simulate_swar4_core's
// Sync policy; the block path has its own).
struct WarpSync {
    // the four conditions' priority maxima over the warp, as two 16-bit pairs
    __device__ __forceinline__ void max4(uint32_t m01, uint32_t m23, uint32_t &P01,
                                         uint32_t &P23) const
    {
        const uint32_t p0 = __reduce_max_sync(kFull, m01 & 0xffffu);
        const uint32_t p1 = __reduce_max_sync(kFull, m01 >> 16);
        const uint32_t p2 = __reduce_max_sync(kFull, m23 & 0xffffu);
        const uint32_t p3 = __reduce_max_sync(kFull, m23 >> 16);
        P01 = prmt(p0, p1, 0x5410u);
        P23 = prmt(p2, p3, 0x5410u);
    }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
    __device__ __forceinline__ uint32_t sum(uint32_t v) const { return __reduce_add_sync(kFull, v); }
    // the state codes of the thread's nodes, where the gather reads them
    template <int NPL, bool SMEM_FMT>
    __device__ __forceinline__ void store_codes(uint8_t *p, const uint32_t (&s4)[NPL], int) const
    {
        store_state_codes<NPL, SMEM_FMT>(p, s4);
    }
    // Error of a time point (Section 2.3) from the compact entry words, read
    // where they are used (nothing is fetched ahead).
    struct Ahead {};
    template <int NPL>
    __device__ __forceinline__ Ahead fetch_obs(const DevNet &, int, int, int) const
    {
        return {};
    }
    template <int NPL, bool>
    __device__ __forceinline__ uint32_t error(const Ahead &, const uint32_t (&s4)[NPL],
                                              const DevNet &net, int g, int tau, int lane,
                                              int) const
    {
        uint32_t w[NPL];
        load_obs<NPL>(w, net.obs + (((size_t)g * net.T + tau) * 32 + lane) * NPL);
        uint32_t e = 0;
#pragma unroll
        for (int k = 0; k < NPL; ++k) e = entry_error(s4[k], w[k], e);
        return e;
    }
};

// The byte-SIMD simulation, shared by the register-table and the
// shared-memory-table instances; `gather(k)` returns slot k's biased image
// bytes (128 + K per condition) from the instance's table words.  A chain's
// nodes sit on LANES threads (a warp, or the block of the block path), whose
// maxima, barriers and score sum come from `sync`.  EARLY reduces over one
// warp and is for LANES = 32 only.
template <int NPL, bool SMEM_FMT, bool EARLY, int LANES = 32, class Gather,
          class Sync = WarpSync>
__device__ __forceinline__ int32_t simulate_swar4_core(const int32_t (&u)[NPL],
                                                       const int32_t (&m1)[NPL],
                                                       const int32_t (&d2)[NPL],
                                                       const DevNet &net, uint8_t *sm,
                                                       uint32_t base, int lane, uint8_t *traj,
                                                       int32_t limit, Gather gather,
                                                       Sync sync = Sync())
{
    static_assert(!EARLY || LANES == 32, "early rejection reduces over one warp");
    const int T = net.T;
    uint8_t *my_codes = sm + base + 2 * lane * NPL;
    uint32_t U2[NPL], CM[NPL];
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
        U2[k] = (uint32_t)u[k] * 0x00010001u;
        CM[k] = (uint32_t)(128 - m1[k]) * kB1;
    }
    uint32_t score = 0;
    for (int g = 0; g < net.G; ++g) {
        uint32_t s4[NPL], cu[NPL], cd[NPL], ua01[NPL], ua23[NPL], mov[NPL];
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
            const size_t q = (size_t)g * LANES * NPL + lane * NPL + k;
            s4[k] = __ldg(net.init_s4 + q);
            mov[k] = __ldg(net.movable + q);
            cu[k] = 0;
            cd[k] = 0;
            ua01[k] = U2[k];
            ua23[k] = U2[k];
        }
        sync.template store_codes<NPL, SMEM_FMT>(my_codes, s4, lane);
        const int ncg = min(net.C - 4 * g, 4);
        for (int tau = 0; tau < T; ++tau) {
            // the entry words of this time point, fetched ahead of the update
            // step where the policy does so
            const auto ahead = sync.template fetch_obs<NPL>(net, g, tau, lane);
            if (net.async && tau > 0) {
                // asynchronous scheme: only the step's selected node may move
                const uint32_t *mt =
                    net.movable_t + ((size_t)(g * T + tau) * LANES + lane) * NPL;
#pragma unroll
                for (int k = 0; k < NPL; ++k) mov[k] = __ldg(mt + k);
            }
            if (tau > 0) {
                uint32_t acc[NPL];
                if constexpr (gathers_pairs<Gather>::value) {
                    static_assert(NPL % 2 == 0, "pairs of slots");
#pragma unroll
                    for (int k = 0; k < NPL; k += 2) gather.pair(k, acc[k], acc[k + 1]);
                } else {
#pragma unroll
                    for (int k = 0; k < NPL; ++k) acc[k] = gather(k);
                }
                uint32_t sn[NPL], pr01[NPL], pr23[NPL], elm[NPL];
                uint32_t m01 = 0, m23 = 0;
#pragma unroll
                for (int k = 0; k < NPL; ++k) {
                    const uint32_t a = acc[k];
                    const uint32_t tgt = target4(a);
                    const uint32_t dp = tgt + 2 * kB1 - s4[k];
                    const uint32_t up = (dp + 0x7D7D7D7Du) & kH;
                    const uint32_t dn = ~(dp + 0x7E7E7E7Eu) & kH;
                    cu[k] = (cu[k] + kB1) & prmt(up, 0u, 0xBA98u);
                    cd[k] = (cd[k] + kB1) & prmt(dn, 0u, 0xBA98u);
                    const uint32_t el = ((cu[k] + CM[k]) | (cd[k] + CM[k])) & mov[k];
                    elm[k] = prmt(el, 0u, 0xBA98u);
                    sn[k] = d2[k] ? tgt : s4[k] + (up >> 7) - (dn >> 7);
                    pr01[k] = ua01[k] & prmt(el, 0u, 0x9988u);
                    pr23[k] = ua23[k] & prmt(el, 0u, 0xBBAAu);
                    m01 = max_u16x2(m01, pr01[k]);
                    m23 = max_u16x2(m23, pr23[k]);
                }
                uint32_t P01, P23;
                sync.max4(m01, m23, P01, P23);   // the maxima over the chain's nodes
#pragma unroll
                for (int k = 0; k < NPL; ++k) {
                    // bit 15 of a half: the node's priority is below the
                    // maximum (P >= pr in each half and both are below 2^15,
                    // so P - pr neither borrows across halves nor carries out)
                    const uint32_t nz01 = (P01 - pr01[k] + 0x7FFF7FFFu) & 0x80008000u;
                    const uint32_t nz23 = (P23 - pr23[k] + 0x7FFF7FFFu) & 0x80008000u;
                    const uint32_t upd = elm[k] & ~prmt(nz01, nz23, 0xFDB9u);
                    s4[k] = (s4[k] & ~upd) | (sn[k] & upd);
                    cu[k] &= ~upd;
                    cd[k] &= ~upd;
                    const uint32_t u01 = prmt(upd, 0u, 0x9988u), u23 = prmt(upd, 0u, 0xBBAAu);
                    ua01[k] = ((ua01[k] + U2[k]) & ~u01) | (U2[k] & u01);
                    ua23[k] = ((ua23[k] + U2[k]) & ~u23) | (U2[k] & u23);
                }
                sync.template store_codes<NPL, SMEM_FMT>(my_codes, s4, lane);
            }
            sync.sync();
            // error at this time point
            score += sync.template error<NPL, SMEM_FMT>(ahead, s4, net, g, tau, lane, ncg);
            if (EARLY && (tau & 3) == 3) {
                // exact early rejection: the partial score never decreases
                const uint32_t tot = __reduce_add_sync(kFull, score) >> 2;
                if (tot > (uint32_t)limit) return (int32_t)tot;
            }
            if (traj) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (c >= ncg) break;
                    const int cc = 4 * g + c;
#pragma unroll
                    for (int k = 0; k < NPL; ++k) {
                        const int i = net.q_node[lane * NPL + k];
                        if (i >= 0)
                            traj[((size_t)cc * T + tau) * net.N + i] =
                                (uint8_t)((s4[k] >> (8 * c)) & 0xffu);
                    }
                }
            }
        }
        sync.sync();
    }
    return (int32_t)(sync.sum(score) >> 2);   // quarter units (entry_error)
}

// The register-table instance: table words in registers (rn_device.cuh format,
// state-code nibble s), gathered in groups of 4 per slot.
template <int NPL, int D0, int D1>
__device__ __forceinline__ int32_t simulate_swar4(const Regs<NPL, D0, D1> &R, const DevNet &net,
                                                  uint8_t *sm, uint32_t base, int lane,
                                                  uint8_t *traj, int32_t limit)
{
    auto gather = [&](int k) -> uint32_t {
        if (k == 0)
            return image<D0>(R.lut0, net.D[0], base, sm, kImage0 - 0x04040404u * groups4(net.D[0]));
        if constexpr (NPL > 1)
            return image<D1>(R.lutr[k - 1], net.D[k], base, sm,
                             kImage0 - 0x04040404u * groups4(net.D[k]));
        return 0u;
    };
    // the early-rejection check lives only in the instance that needs it
    if (limit == INT32_MAX)
        return simulate_swar4_core<NPL, false, false>(R.u, R.m1, R.d2, net, sm, base, lane, traj,
                                                      limit, gather);
    return simulate_swar4_core<NPL, false, true>(R.u, R.m1, R.d2, net, sm, base, lane, traj,
                                                 limit, gather);
}

// The scalar update (groups of CG conditions, one integer per node and
// condition), used when a network has a single condition.  EARLY compiles the
// early-rejection check against `limit`.
template <int NPL, int CG, int D0, int D1, bool EARLY>
__device__ __forceinline__ int32_t simulate_scalar(const Regs<NPL, D0, D1> &R, const DevNet &net,
                                                   uint8_t *sm, uint32_t base, int lane,
                                                   uint8_t *traj, int32_t limit)
{
    const int T = net.T;
    uint8_t *my_codes = sm + base + 2 * lane * NPL;
    uint32_t score = 0;
    for (int g = 0; g < net.G; ++g) {
        uint32_t code[NPL];
        load_codes<NPL>(code, net.init_code + (size_t)g * 32 * NPL + lane * NPL);
        const uint32_t outb = net.out_bits[g * 32 + lane];
        int32_t s[NPL][CG], run[NPL][CG], ua[NPL][CG];
#pragma unroll
        for (int k = 0; k < NPL; ++k)
#pragma unroll
            for (int c = 0; c < CG; ++c) {
                s[k][c] = (code[k] >> (4 * c)) & 0xf;
                run[k][c] = 0;
                // synchronous scheme: u = 0 and every eligible node at priority 1
                ua[k][c] = ((outb >> (k * CG + c)) & 1u) ? kOutUA : (R.u[k] | net.sync);
            }
        store_codes<NPL>(my_codes, code);
        int ncg = net.C - g * CG;
        if (ncg > CG) ncg = CG;
        for (int tau = 0; tau < T; ++tau) {
            if (tau > 0) {
                uint32_t acc[NPL];
                images<NPL, D0, D1>(acc, R, net, base, sm);
#pragma unroll
                for (int c = 0; c < CG; ++c) {
                    int32_t pr[NPL], sn[NPL], pmax = 0;
#pragma unroll
                    for (int k = 0; k < NPL; ++k) {
                        const int32_t lo = 4 * groups4(net.D[k]);
                        const int32_t kb = (int32_t)((acc[k] >> (8 * c)) & 0xffu);
                        const int32_t tgt = min(max(kb, lo), lo + 2) - lo;
                        const int32_t diff = tgt - s[k][c];
                        const int32_t sg = min(max(diff, -1), 1);
                        const int32_t t = max(run[k][c] * sg + 1, 1);
                        run[k][c] = t * sg;
                        pr[k] = abs(run[k][c]) >= R.m1[k] ? ua[k][c] : 0;
                        sn[k] = R.d2[k] ? tgt : s[k][c] + sg;
                    }
                    if (net.async && g * CG + c < net.C) {
                        // asynchronous scheme: only the step's selected node may move
                        const int sel = __ldg(net.async_sel + (size_t)(g * CG + c) * T + tau);
#pragma unroll
                        for (int k = 0; k < NPL; ++k)
                            if (net.q_node[lane * NPL + k] != sel) pr[k] = 0;
                    }
#pragma unroll
                    for (int k = 0; k < NPL; ++k) pmax = max(pmax, pr[k]);
                    pmax = __reduce_max_sync(kFull, pmax);
#pragma unroll
                    for (int k = 0; k < NPL; ++k) {
                        const bool upd = pr[k] == pmax && pr[k] > 0;
                        s[k][c] = upd ? sn[k] : s[k][c];
                        run[k][c] = upd ? 0 : run[k][c];
                        ua[k][c] = upd ? (R.u[k] | net.sync) : ua[k][c] + R.u[k];
                    }
                }
#pragma unroll
                for (int k = 0; k < NPL; ++k) {
                    uint32_t cd = 0;
#pragma unroll
                    for (int c = 0; c < CG; ++c) cd |= (uint32_t)s[k][c] << (4 * c);
                    code[k] = cd;
                }
                store_codes<NPL>(my_codes, code);
            }
            __syncwarp();
            // error of the lane's nodes at this time point: sum W |s - R| from the
            // entry tables (byte b = W |b - R|)
#pragma unroll
            for (int c = 0; c < CG; ++c) {
                if (c >= ncg) break;
                const int cc = g * CG + c;
                uint32_t w[NPL];
                load_obs<NPL>(w, net.obs + (((size_t)cc * T + tau) * 32 + lane) * NPL);
                uint32_t t = 0;
#pragma unroll
                for (int k = 0; k < NPL; ++k) t += __byte_perm(w[k], 0u, (uint32_t)s[k][c]);
                score += t & 0xffu;
                if (traj) {
#pragma unroll
                    for (int k = 0; k < NPL; ++k) {
                        const int i = net.q_node[lane * NPL + k];
                        if (i >= 0) traj[((size_t)cc * T + tau) * net.N + i] = (uint8_t)s[k][c];
                    }
                }
            }
            if (EARLY && (tau & 3) == 3) {
                // exact early rejection: the partial score never decreases
                const uint32_t tot = __reduce_add_sync(kFull, score);
                if (tot > (uint32_t)limit) return (int32_t)tot;
            }
        }
        __syncwarp();
    }
    return (int32_t)__reduce_add_sync(kFull, score);
}

// Simulate(x) of Table 1 for the warp's vector: every condition, every time
// step (Sections 2.1-2.2), scored against the entry tables (Section 2.3).
// Returns y in every lane.  With traj != null, writes S to traj[C][T][N].
// `base` is the warp's 256-byte-aligned offset of its state codes in `sm`.
// With limit < INT32_MAX the simulation may stop early and return any value
// above `limit` once the partial score (which never decreases) exceeds it.
template <int NPL, int CG, int D0, int D1>
__device__ __forceinline__ int32_t simulate(const Regs<NPL, D0, D1> &R, const DevNet &net,
                                            uint8_t *sm, uint32_t base, int lane, uint8_t *traj,
                                            int32_t limit = INT32_MAX)
{
    if constexpr (CG == 4) return simulate_swar4<NPL, D0, D1>(R, net, sm, base, lane, traj, limit);
    if (limit == INT32_MAX)
        return simulate_scalar<NPL, CG, D0, D1, false>(R, net, sm, base, lane, traj, limit);
    return simulate_scalar<NPL, CG, D0, D1, true>(R, net, sm, base, lane, traj, limit);
}

}  // namespace rn
