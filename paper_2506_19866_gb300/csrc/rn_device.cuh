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

constexpr int kMaxSlots = 4;          // nodes per lane in the register-table kernels
constexpr uint32_t kFull = 0xffffffffu;
constexpr int32_t kOutUA = -(1 << 22);   // priority seed of a node that never moves

// Network as the kernels see it (all pointers are device memory).
struct DevNet {
    int32_t N, E, P, n_free;
    int32_t C, T, G;                    // conditions, time points, condition groups
    int32_t npl, cg, dtab;              // nodes per lane, conditions per group, table stride
    int32_t D[kMaxSlots];               // padded in-degree of each slot
    const int32_t *edge_id;             // [npl][dtab][32] edge index or -1 (padding)
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
struct DevSched {
    int64_t g0, g1;
    int64_t iters;                      // proposals per level
    int64_t level0;                     // level of thr_off[0]
    int32_t reset_to_best;
    const int32_t *thr_off;             // [levels] start of the level's table
    const int32_t *thr_len;             // [levels] D_l: largest dE with a nonzero threshold
    const uint32_t *thr;                // entries for dE = 1 .. D_l
};

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
        uint32_t w = 0x00040404u | ((uint32_t)(2 * (lane * NPL + k)) << 24);   // padding: f = 0
        if (d < net.D[k]) {
            const int e = net.edge_id[(k * net.dtab + d) * 32 + lane];
            if (e >= 0) w = edge_word(x[e], x[E + e], x[2 * E + e], net.edge_q2[e]);
        }
        word = w;
    });
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
        const int i = net.q_node[lane * NPL + k];
        if (i >= 0) {
            R.u[k] = x[3 * E + i];
            R.m1[k] = x[3 * E + N + i] + 1;
            R.d2[k] = x[3 * E + 2 * N + i] == 2;
        } else {
            R.u[k] = 1;
            R.m1[k] = 1;
            R.d2[k] = 0;
        }
    }
}

// Biased image terms of the slot's node for the CG conditions, one byte each:
// sum over its D in-edges.  D is warp uniform: the jump into the unrolled
// sequence does not diverge.
template <int DC>
__device__ __forceinline__ uint32_t image(const uint32_t (&lut)[DC], int D, uint32_t base,
                                          const uint8_t *sm)
{
    uint32_t acc = 0;
#define RN_EDGE(dd)                                                                    \
    case (dd) + 1:                                                                     \
        if constexpr (DC > (dd)) {                                                     \
            const uint32_t a = __byte_perm(lut[dd], base, 0x7653u);                    \
            acc += __byte_perm(lut[dd], 0u, (uint32_t)(*(const uint16_t *)(sm + a)));  \
        }                                                                              \
        [[fallthrough]];
    switch (D) {
        RN_EDGE(15) RN_EDGE(14) RN_EDGE(13) RN_EDGE(12) RN_EDGE(11) RN_EDGE(10) RN_EDGE(9)
        RN_EDGE(8) RN_EDGE(7) RN_EDGE(6) RN_EDGE(5) RN_EDGE(4) RN_EDGE(3) RN_EDGE(2)
        RN_EDGE(1) RN_EDGE(0)
    default:
        break;
    }
#undef RN_EDGE
    return acc;
}

template <int NPL, int D0, int D1>
__device__ __forceinline__ void images(uint32_t (&acc)[NPL], const Regs<NPL, D0, D1> &R,
                                       const DevNet &net, uint32_t base, const uint8_t *sm)
{
    acc[0] = image<D0>(R.lut0, net.D[0], base, sm);
#pragma unroll
    for (int k = 1; k < NPL; ++k) acc[k] = image<D1>(R.lutr[k - 1], net.D[k], base, sm);
}

template <int NPL>
__device__ __forceinline__ void store_codes(uint8_t *p, const uint32_t (&code)[NPL])
{
    if constexpr (NPL == 1) {
        *reinterpret_cast<uint16_t *>(p) = (uint16_t)code[0];
    } else if constexpr (NPL == 2) {
        *reinterpret_cast<uint32_t *>(p) = code[0] | (code[1] << 16);
    } else {
        *reinterpret_cast<uint2 *>(p) = make_uint2(code[0] | (code[1] << 16),
                                                   code[2] | (code[3] << 16));
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
    if constexpr (NPL == 4) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(ob));
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    } else if constexpr (NPL == 2) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(ob));
        w[0] = v.x; w[1] = v.y;
    } else {
        w[0] = __ldg(ob);
    }
}

// Simulate(x) of Table 1 for the warp's vector: every condition, every time
// step (Sections 2.1-2.2), scored against the entry tables (Section 2.3).
// Returns y in every lane.  With traj != null, writes S to traj[C][T][N].
// `base` is the warp's 256-byte-aligned offset of its state codes in `sm`.
template <int NPL, int CG, int D0, int D1>
__device__ __forceinline__ int32_t simulate(const Regs<NPL, D0, D1> &R, const DevNet &net,
                                            uint8_t *sm, uint32_t base, int lane, uint8_t *traj)
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
                ua[k][c] = ((outb >> (k * CG + c)) & 1u) ? kOutUA : R.u[k];
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
                        const int32_t lo = 4 * net.D[k];
                        const int32_t kb = (int32_t)((acc[k] >> (8 * c)) & 0xffu);
                        const int32_t tgt = min(max(kb, lo), lo + 2) - lo;
                        const int32_t diff = tgt - s[k][c];
                        const int32_t sg = min(max(diff, -1), 1);
                        const int32_t t = max(run[k][c] * sg + 1, 1);
                        run[k][c] = t * sg;
                        pr[k] = abs(run[k][c]) >= R.m1[k] ? ua[k][c] : 0;
                        sn[k] = R.d2[k] ? tgt : s[k][c] + sg;
                        pmax = max(pmax, pr[k]);
                    }
                    pmax = __reduce_max_sync(kFull, pmax);
#pragma unroll
                    for (int k = 0; k < NPL; ++k) {
                        const bool upd = pr[k] == pmax && pr[k] > 0;
                        s[k][c] = upd ? sn[k] : s[k][c];
                        run[k][c] = upd ? 0 : run[k][c];
                        ua[k][c] = upd ? R.u[k] : ua[k][c] + R.u[k];
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
        }
        __syncwarp();
    }
    return (int32_t)__reduce_add_sync(kFull, score);
}

}  // namespace rn
