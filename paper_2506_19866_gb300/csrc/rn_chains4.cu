// rn_chains4.cu -- annealing of single-condition networks with four chains per
// warp in the byte lanes.
//
// A network with one time course (the paper's own case: one condition) leaves
// three of the four byte lanes of the condition-SIMD simulation idle, so its
// warps ran a scalar update instead.  Here one warp advances four chains of
// the network together: byte c of every per-node word belongs to chain 4q + c.
// The chains share the topology, the time course and the state-code
// addresses, but not the parameters, so each chain keeps its own register
// table words (byte 3, the source's code address, only in chain 0's word;
// zero in the others), and the per-node constants u, m + 1 and d = 2 are
// per byte.  The image of a node's slot adds, per in-edge, two PRMTs of the
// four chains' words selected by the source's state code, whose nibbles are
// (s0, 4 + s1, s2, 4 + s3) in this layout; the priority update is the
// byte-SIMD update of the condition path (Section 2.2) with per-byte
// constants; the error of a node at a time point is one PRMT of its
// single-condition error word (bytes W |s - R| for s = 0, 1, 2) by the same
// code (Section 2.3).  Each chain proposes, accepts and rolls back on its own
// (Table 1) with the Philox words of its own chain index, so every chain is
// bit-identical to the one-chain-per-warp run.  A work item is a chunk of
// steps of a quad of chains; the last quad may be partly empty.
#include "rn_kernels.cuh"
#include "rn_screen.h"

namespace rn {
namespace {

template <int NPL, int D0, int D1>
struct Regs4 {
    uint32_t lut0[4][D0];
    uint32_t lutr[4][NPL > 1 ? NPL - 1 : 1][D1];
    uint32_t U01[NPL], U23[NPL];   // speed u of chains 0, 1 (2, 3) as 16-bit halves
    uint32_t CM[NPL];              // byte c: 128 - (m + 1) of chain c
    uint32_t D2[NPL];              // byte c: 0xff where d = 2 in chain c
};

// Undo record of chain c's changed entry, kept by its owner lane only: the
// entry (kind << 16 | slot << 10 | slot * 32 + edge column) and its old value.
struct Undo4 {
    uint32_t what[4], val[4];
};

// Visit chain c's table word of (slot k, edge d) with compile-time k and d.
template <int NPL, int D0, int D1, typename F>
__device__ __forceinline__ void for_each_word4(Regs4<NPL, D0, D1> &R, int c, F f)
{
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
        if (cc != c) continue;
#pragma unroll
        for (int d = 0; d < D0; ++d) f(0, d, R.lut0[cc][d]);
#pragma unroll
        for (int k = 1; k < NPL; ++k)
#pragma unroll
            for (int d = 0; d < D1; ++d) f(k, d, R.lutr[cc][k - 1][d]);
    }
}

__device__ __forceinline__ void put_byte(uint32_t &w, int c, uint32_t b)
{
    w = (w & ~(0xffu << (8 * c))) | ((b & 0xffu) << (8 * c));
}

__device__ __forceinline__ void put_half(uint32_t &w, int h, uint32_t v)
{
    w = (w & ~(0xffffu << (16 * h))) | ((v & 0xffffu) << (16 * h));
}

// Per-node constants of chain c from its x.
template <int NPL, int D0, int D1>
__device__ __forceinline__ void load_node_consts(Regs4<NPL, D0, D1> &R, const DevNet &net,
                                                 const int8_t *x, int c, int k, int lane)
{
    const int E = net.E, N = net.N;
    const int i = net.q_node[lane * NPL + k];
    uint32_t u = 1, m1 = 1, d2 = 0;
    if (i >= 0) {
        u = net.sync ? 0u : (uint32_t)x[3 * E + i];
        m1 = (uint32_t)x[3 * E + N + i] + 1u;
        d2 = x[3 * E + 2 * N + i] == 2 ? 0xffu : 0u;
    }
    if (c < 2) put_half(R.U01[k], c, u);
    else put_half(R.U23[k], c - 2, u);
    put_byte(R.CM[k], c, 128u - m1);
    put_byte(R.D2[k], c, d2);
}

// Tables and constants of the four chains (x of chain c at xs[c]).
template <int NPL, int D0, int D1>
__device__ __forceinline__ void load_regs4(Regs4<NPL, D0, D1> &R, const DevNet &net,
                                           int8_t *const (&xs)[4], int lane)
{
    const int E = net.E;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int8_t *x = xs[c];
        for_each_word4<NPL, D0, D1>(R, c, [&](int k, int d, uint32_t &word) {
            // padding reads a valid code (that of node 2 lane, or the lane's own
            // node with one node per lane) and adds 4 in every byte
            uint32_t a = (uint32_t)((NPL == 1 ? 2 : 4) * lane);
            uint32_t w = 0x00040404u;
            if (d < net.D[k]) {
                const int e = net.edge_id[(k * net.dtab + d) * 32 + lane];
                if (e >= 0) {
                    w = edge_word(x[e], x[E + e], x[2 * E + e], 0u);
                    a = net.edge_q2[e];
                } else {
                    a = (uint32_t)(-1 - e);
                }
            }
            word = c == 0 ? (w | (a << 24)) : w;
        });
#pragma unroll
        for (int k = 0; k < NPL; ++k) load_node_consts(R, net, x, c, k, lane);
    }
}

// Biased image bytes of slot k for the four chains (byte c: 127 + K of chain c
// after the kImage0 - 4 D4 start), from the four chains' words and the
// sources' codes.
template <int DC>
__device__ __forceinline__ uint32_t image4(const uint32_t (&l0)[DC], const uint32_t (&l1)[DC],
                                           const uint32_t (&l2)[DC], const uint32_t (&l3)[DC],
                                           int D, uint32_t base, const uint8_t *sm)
{
    uint32_t acc = kImage0 - 0x04040404u * (uint32_t)groups4(D);
#pragma unroll
    for (int g = 0; g < DC; g += 4) {
        if (g < D) {
            uint32_t code[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                code[i] = *(const uint16_t *)(sm + __byte_perm(l0[g + i], base, 0x7653u));
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t s01 = (code[i] & 0x00ffu) | 0x7700u;   // (s0, 4 + s1, zero, zero)
                const uint32_t s23 = (code[i] & 0xff00u) | 0x0033u;   // (zero, zero, s2, 4 + s3)
                acc += __byte_perm(l0[g + i], l1[g + i], s01) + __byte_perm(l2[g + i], l3[g + i], s23);
            }
        }
    }
    return acc;
}

// Simulate() of Table 1 for the four chains: their scores y into y[4]
// (warp-uniform).  One condition (G = 1); error words of the single-condition
// layout, [T][32][NPL] with byte b = W |b - R|.
template <int NPL, int D0, int D1>
__device__ __forceinline__ void simulate4(const Regs4<NPL, D0, D1> &R, const DevNet &net,
                                          uint8_t *sm, uint32_t base, int lane, int32_t (&y)[4])
{
    const int T = net.T;
    uint8_t *my_codes = sm + base + 2 * lane * NPL;
    uint32_t s4[NPL], cu[NPL], cd[NPL], ua01[NPL], ua23[NPL], mov[NPL], code[NPL];
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
        const int q = lane * NPL + k;
        s4[k] = (__ldg(net.init_s4 + q) & 0xffu) * kB1;
        mov[k] = (__ldg(net.movable + q) & 0x80u) ? kH : 0u;
        cu[k] = 0;
        cd[k] = 0;
        ua01[k] = R.U01[k];
        ua23[k] = R.U23[k];
        code[k] = state_code<false>(s4[k]) + 0x4040u;
    }
    store_codes<NPL>(my_codes, code);
    uint32_t e01 = 0, e23 = 0;   // per-chain error sums as 16-bit halves
    for (int tau = 0; tau < T; ++tau) {
        // this time point's error words, loaded before the update step so that
        // their latency overlaps it (with two nodes per lane; one node per lane
        // loads them where they are used, which keeps its register allocation
        // free of spills)
        uint32_t ew[NPL];
        if constexpr (NPL == 2) {
#pragma unroll
            for (int k = 0; k < NPL; ++k)
                ew[k] = __ldg(net.obs + ((size_t)tau * 32 + lane) * NPL + k);
        }
        if (tau > 0) {
            uint32_t acc[NPL];
            acc[0] = image4<D0>(R.lut0[0], R.lut0[1], R.lut0[2], R.lut0[3], net.D[0], base, sm);
            if constexpr (NPL > 1) {
#pragma unroll
                for (int k = 1; k < NPL; ++k)
                    acc[k] = image4<D1>(R.lutr[0][k - 1], R.lutr[1][k - 1], R.lutr[2][k - 1],
                                        R.lutr[3][k - 1], net.D[k], base, sm);
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
                const uint32_t el = ((cu[k] + R.CM[k]) | (cd[k] + R.CM[k])) & mov[k];
                elm[k] = prmt(el, 0u, 0xBA98u);
                const uint32_t step1 = s4[k] + (up >> 7) - (dn >> 7);
                sn[k] = (tgt & R.D2[k]) | (step1 & ~R.D2[k]);
                pr01[k] = ua01[k] & prmt(el, 0u, 0x9988u);
                pr23[k] = ua23[k] & prmt(el, 0u, 0xBBAAu);
                m01 = max_u16x2(m01, pr01[k]);
                m23 = max_u16x2(m23, pr23[k]);
            }
            const uint32_t p0 = __reduce_max_sync(kFull, m01 & 0xffffu);
            const uint32_t p1 = __reduce_max_sync(kFull, m01 >> 16);
            const uint32_t p2 = __reduce_max_sync(kFull, m23 & 0xffffu);
            const uint32_t p3 = __reduce_max_sync(kFull, m23 >> 16);
            const uint32_t P01 = prmt(p0, p1, 0x5410u), P23 = prmt(p2, p3, 0x5410u);
#pragma unroll
            for (int k = 0; k < NPL; ++k) {
                const uint32_t nz01 = ((pr01[k] ^ P01) + 0x7FFF7FFFu) & 0x80008000u;
                const uint32_t nz23 = ((pr23[k] ^ P23) + 0x7FFF7FFFu) & 0x80008000u;
                const uint32_t upd = elm[k] & ~prmt(nz01, nz23, 0xFDB9u);
                s4[k] = (s4[k] & ~upd) | (sn[k] & upd);
                cu[k] &= ~upd;
                cd[k] &= ~upd;
                const uint32_t u01 = prmt(upd, 0u, 0x9988u), u23 = prmt(upd, 0u, 0xBBAAu);
                ua01[k] = ((ua01[k] + R.U01[k]) & ~u01) | (R.U01[k] & u01);
                ua23[k] = ((ua23[k] + R.U23[k]) & ~u23) | (R.U23[k] & u23);
                code[k] = state_code<false>(s4[k]) + 0x4040u;
            }
            store_codes<NPL>(my_codes, code);
        }
        __syncwarp();
        // error at this time point: byte c = W |s_c - R| summed over the lane's nodes
        uint32_t eb = 0;
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
            if constexpr (NPL != 2) ew[k] = __ldg(net.obs + ((size_t)tau * 32 + lane) * NPL + k);
            eb += __byte_perm(ew[k], ew[k], code[k]);
        }
        e01 += __byte_perm(eb, 0u, 0x4140u);
        e23 += __byte_perm(eb, 0u, 0x4342u);
    }
    __syncwarp();
    y[0] = (int32_t)__reduce_add_sync(kFull, e01 & 0xffffu);
    y[1] = (int32_t)__reduce_add_sync(kFull, e01 >> 16);
    y[2] = (int32_t)__reduce_add_sync(kFull, e23 & 0xffffu);
    y[3] = (int32_t)__reduce_add_sync(kFull, e23 >> 16);
}

// Chain c's table entry or node constant (parameter kind `kind`, index idx in
// its block of x) takes the candidate's value (owner lane only), with an undo
// record.  Returns whether this lane is the owner.
template <int NPL, int D0, int D1>
__device__ __forceinline__ bool change4_ki(Regs4<NPL, D0, D1> &R, Undo4 &U, const DevNet &net,
                                           const int8_t *x, int c, int lane, int kind, int idx,
                                           int v)
{
    const int E = net.E;
    if (kind < 3) {
        const int pos = net.edge_pos[idx];
        if (lane != (pos >> 16)) return false;
        int w = x[idx], p = x[E + idx], t = x[2 * E + idx];
        if (kind == 0) w = v; else if (kind == 1) p = v; else t = v;
        const int kd = ((pos >> 8) & 0xff) * 32 + (pos & 0xff);
        uint32_t old = 0;
        for_each_word4<NPL, D0, D1>(R, c, [&](int k, int d, uint32_t &word) {
            old = (k * 32 + d == kd) ? word : old;
        });
        const uint32_t nw = edge_word(w, p, t, 0u) | (old & 0xff000000u);
        for_each_word4<NPL, D0, D1>(R, c, [&](int k, int d, uint32_t &word) {
            word = (k * 32 + d == kd) ? nw : word;
        });
#pragma unroll
        for (int cc = 0; cc < 4; ++cc)
            if (cc == c) { U.what[cc] = (uint32_t)kd; U.val[cc] = old; }
        return true;
    }
    const int q = net.node_q[idx];
    if (lane != q / NPL) return false;
    const int slot = q - (q / NPL) * NPL;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
        if (cc != c) continue;
        U.what[cc] = ((uint32_t)kind << 16) | ((uint32_t)slot << 10);
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
            if (k != slot) continue;
            if (kind == 3) {
                uint32_t &Uk = cc < 2 ? R.U01[k] : R.U23[k];
                U.val[cc] = Uk;
                put_half(Uk, cc & 1, net.sync ? 0u : (uint32_t)v);
            } else if (kind == 4) {
                U.val[cc] = R.CM[k];
                put_byte(R.CM[k], cc, 127u - (uint32_t)v);
            } else {
                U.val[cc] = R.D2[k];
                put_byte(R.D2[k], cc, v == 2 ? 0xffu : 0u);
            }
        }
    }
    return true;
}

// The same for parameter j of x.
template <int NPL, int D0, int D1>
__device__ __forceinline__ bool change4(Regs4<NPL, D0, D1> &R, Undo4 &U, const DevNet &net,
                                        const int8_t *x, int c, int lane, int j, int v)
{
    const int E = net.E, N = net.N;
    int kind, idx;
    param_kind(j, E, N, kind, idx);
    return change4_ki<NPL, D0, D1>(R, U, net, x, c, lane, kind, idx, v);
}

template <int NPL, int D0, int D1>
__device__ __forceinline__ void undo4(Regs4<NPL, D0, D1> &R, const Undo4 &U, int c)
{
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
        if (cc != c) continue;
        const uint32_t kind = U.what[cc] >> 16, ov = U.val[cc];
        if (kind == 0) {
            const int kd = (int)(U.what[cc] & 0x3ffu);
            for_each_word4<NPL, D0, D1>(R, cc, [&](int k, int d, uint32_t &word) {
                word = (k * 32 + d == kd) ? ov : word;
            });
            continue;
        }
        // the constants of the four chains share registers: restore only
        // chain cc's byte (half for u), since another chain's change to the
        // same node may have been accepted in the same step
        const int slot = (int)((U.what[cc] >> 10) & 0x3fu);
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
            if (k != slot) continue;
            if (kind == 3) put_half(cc < 2 ? R.U01[k] : R.U23[k], cc & 1, ov >> (16 * (cc & 1)));
            else if (kind == 4) put_byte(R.CM[k], cc, ov >> (8 * cc));
            else put_byte(R.D2[k], cc, ov >> (8 * cc));
        }
    }
}

// Steps [g_lo, g_hi) of the chains 4 quad .. 4 quad + 3 (those below ch.n),
// their state in and out of global memory through L2, then the quad's chunk
// counter is published.  `region`: chain c's x at c * per_chain, its two
// constraint counters after it; `cnt`: the four chains' accepted, uphill and
// null counts of the chunk (lane 0 keeps them).
template <int NPL, int D0, int D1>
__device__ __forceinline__ void run_chunk4(const DevNet &net, const DevChains &ch,
                                           const DevSched &sc, uint8_t *sm, uint32_t base,
                                           uint8_t *region, uint32_t per_chain, int32_t *cnt,
                                           int quad, int64_t g_lo, int64_t g_hi,
                                           int32_t *done_flag, int done_value, int lane)
{
    Regs4<NPL, D0, D1> R;
    Undo4 U;
    const uint32_t nr = round16((uint32_t)net.N);
    const int n_here = min(4, ch.n - 4 * quad);   // chains of this quad
    auto xs = [&](int c) { return reinterpret_cast<int8_t *>(region + (uint32_t)c * per_chain); };
    auto onz = [&](int c) { return region + (uint32_t)c * per_chain + (uint32_t)ch.pstride; };
    auto pin = [&](int c) { return onz(c) + nr; };
    auto load_rows = [&](const int8_t *rows) {
        // an empty chain of the last quad runs on a copy of chain 4 quad
#pragma unroll
        for (int c = 0; c < 4; ++c)
            warp_load_cg(xs(c), rows + (size_t)(4 * quad + (c < n_here ? c : 0)) * ch.pstride,
                         ch.pstride, lane);
        __syncwarp();
        int8_t *const x4[4] = {xs(0), xs(1), xs(2), xs(3)};
        load_regs4<NPL, D0, D1>(R, net, x4, lane);
#pragma unroll
        for (int c = 0; c < 4; ++c) count_constraints(net, xs(c), onz(c), pin(c), lane);
        __syncwarp();
    };
    load_rows(ch.x_cur);
    int32_t d_cur[4], d_best[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        d_cur[c] = c < n_here ? __ldcg(ch.d_cur + 4 * quad + c) : 0;
        d_best[c] = c < n_here ? __ldcg(ch.d_best + 4 * quad + c) : 0;
    }
    if (lane < 12) cnt[lane] = 0;
    __syncwarp();
    int64_t level = g_lo / sc.iters;
    int64_t in_level = g_lo - level * sc.iters;
    for (int64_t g = g_lo; g < g_hi; ++g) {
        if (in_level == sc.iters) {
            in_level = 0;
            ++level;
        }
        if (sc.reset_to_best && in_level == 0) {
            // Table 1: every level starts from the chain's x_best
            load_rows(ch.x_best);
#pragma unroll
            for (int c = 0; c < 4; ++c) d_cur[c] = d_best[c];
        }
        ++in_level;
        // candidates: lane group c (lanes 8c .. 8c + 7) draws chain c's words
        // and runs its GetCandidate, then every lane takes the four results:
        // cj (parameter), ck (its kind << 28 | index in its block of x), cv (new
        // value | old value << 8), rz (acceptance word); own: bit c when this
        // lane owns chain c's change
        int cj[4], ck[4], cv[4];
        uint32_t rz[4];
        uint32_t has = 0, own = 0;
        {
            const int grp = lane >> 3;
            int j = 0, kind, idx, cur = 0, v = 0, ok = 0;
            uint32_t z = 0;
            if (grp < n_here && net.n_free > 0) {
                const uint4 r = philox(ch.seed, (uint32_t)g, (uint32_t)((uint64_t)g >> 32),
                                       (uint32_t)(4 * quad + grp), 0u);
                z = r.z;
                ok = get_candidate<true>(net, xs(grp), onz(grp), pin(grp), r.x, r.y, j, kind, idx, cur,
                                         v);
            }
            const int packed = ok ? ((v & 0xff) | ((cur & 0xff) << 8)) : -1;
            const int ki = ok ? (kind << 28) | idx : 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                rz[c] = __shfl_sync(kFull, z, 8 * c);
                cj[c] = __shfl_sync(kFull, j, 8 * c);
                ck[c] = __shfl_sync(kFull, ki, 8 * c);
                cv[c] = __shfl_sync(kFull, packed, 8 * c);
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (cv[c] < 0) continue;
            has |= 1u << c;
            if (change4_ki<NPL, D0, D1>(R, U, net, xs(c), c, lane, ck[c] >> 28,
                                        ck[c] & 0x0fffffff, (int8_t)(cv[c] & 0xff)))
                own |= 1u << c;
        }
        if (!has) {
            if (lane == 0)
                for (int c = 0; c < n_here; ++c) cnt[8 + c] += 1;
            continue;
        }
        __syncwarp();
        int32_t y[4];
        simulate4<NPL, D0, D1>(R, net, sm, base, lane, y);
        const int64_t l = level - sc.level0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (c >= n_here) continue;
            if (!(has & (1u << c))) {
                if (lane == 0) cnt[8 + c] += 1;
                continue;
            }
            // Metropolis acceptance against the host-computed threshold table
            const int32_t dE = y[c] - d_cur[c];
            bool accept = dE <= 0;
            if (!accept && dE <= sc.thr_len[l]) accept = rz[c] < __ldg(sc.thr + sc.thr_off[l] + dE - 1);
            if (accept) {
                const int j = cj[c], v = (int8_t)(cv[c] & 0xff), cur = (int8_t)(cv[c] >> 8);
                if (lane == 0) {
                    apply_counters(net, xs(c), onz(c), pin(c), ck[c] >> 28, ck[c] & 0x0fffffff,
                                   cur, v);
                    xs(c)[j] = (int8_t)v;
                    cnt[c] += 1;
                    cnt[4 + c] += dE > 0;
                }
                __syncwarp();
                d_cur[c] = y[c];
                if (y[c] < d_best[c]) {
                    d_best[c] = y[c];
                    warp_store_cg(ch.x_best + (size_t)(4 * quad + c) * ch.pstride, xs(c),
                                  ch.pstride, lane);
                }
            } else if (own & (1u << c)) {
                undo4<NPL, D0, D1>(R, U, c);
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if (c >= n_here) continue;
        const int chain = 4 * quad + c;
        warp_store_cg(ch.x_cur + (size_t)chain * ch.pstride, xs(c), ch.pstride, lane);
        if (lane == 0) {
            __stcg(ch.d_cur + chain, d_cur[c]);
            __stcg(ch.d_best + chain, d_best[c]);
            int64_t *cc = ch.cnt + 3 * (size_t)chain;
            __stcg(cc + 0, __ldcg(cc + 0) + cnt[c]);
            __stcg(cc + 1, __ldcg(cc + 1) + cnt[4 + c]);
            __stcg(cc + 2, __ldcg(cc + 2) + cnt[8 + c]);
        }
    }
    // publish: every lane's stores, then the quad's chunk counter
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicExch(done_flag, done_value);
    __syncwarp();
}

// Shared memory of a warp's four chains: x and the two constraint counters each.
__host__ __device__ inline uint32_t chain4_bytes(int pstride, int N)
{
    return (uint32_t)pstride + 2u * round16((uint32_t)N);
}

// A warp's region: the four chains, then their 12 chunk counters.
__host__ __device__ inline uint32_t chain4_region(int pstride, int N)
{
    return round16(4u * chain4_bytes(pstride, N) + 12u * 4u);
}

template <int NPL, int D0, int D1>
__global__ void __launch_bounds__(128, 3)
    anneal_c4_kernel(DevNet net, DevChains ch, DevSched sc, uint32_t region_bytes)
{
    extern __shared__ __align__(256) uint8_t sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    uint8_t *region = sm + (uint32_t)wpb * kCodeBytesPerWarp + (uint32_t)warp * region_bytes;
    const uint32_t base = (uint32_t)warp * kCodeBytesPerWarp;
    const uint32_t per_chain = chain4_bytes(ch.pstride, net.N);
    const int quads = (ch.n + 3) / 4;
    const int64_t n_items = (int64_t)sc.n_chunks * quads;
    for (;;) {
        unsigned int item = 0;
        if (lane == 0) item = atomicAdd(sc.queue, 1u);
        item = __shfl_sync(kFull, item, 0);
        if ((int64_t)item >= n_items) break;
        const int cj = (int)(item / (unsigned)quads);
        const int quad = (int)(item - (unsigned)cj * (unsigned)quads);
        // chunk cj - 1 of this quad was handed out `quads` items earlier
        if (cj > 0 && !wait_for_chunk(sc.done + quad, cj, sc.err, lane)) return;
        const int64_t g_lo = sc.g0 + (int64_t)cj * sc.chunk;
        const int64_t g_hi = min(sc.g1, g_lo + sc.chunk);
        run_chunk4<NPL, D0, D1>(net, ch, sc, sm, base, region, per_chain,
                                reinterpret_cast<int32_t *>(region + 4u * per_chain), quad, g_lo,
                                g_hi, sc.done + quad, cj + 1, lane);
    }
}

template <int NPL, int D0, int D1>
cudaError_t launch_t(const DevNet &net, const DevChains &ch, const DevSched &sc, int sm_count,
                     cudaStream_t st)
{
    int wpb = 4;
    const uint32_t rb = chain4_region(ch.pstride, net.N);
    size_t smem = (size_t)wpb * (kCodeBytesPerWarp + rb);
    auto kern = anneal_c4_kernel<NPL, D0, D1>;
    cudaError_t err =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wpb * 32, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = sm_count * per_sm;
    const int quads = (ch.n + 3) / 4;
    if (quads > 0 && quads < grid * wpb) {
        // Fewer quads than resident warps: a block of one warp per quad, which
        // the hardware spreads evenly over the SMs.  (In the full grid the
        // quads would go to whichever warps reach the queue first, and one
        // SM could hold several times another's share.)
        wpb = 1;
        grid = quads;
        smem = kCodeBytesPerWarp + rb;
    }
    DevSched s = sc;
    plan_chunks(s, quads, (int64_t)grid * wpb);
    err = cudaMemsetAsync(s.queue, 0, sizeof(unsigned int), st);
    if (err == cudaSuccess) err = cudaMemsetAsync(s.done, 0, sizeof(int32_t) * (size_t)quads, st);
    if (err != cudaSuccess) return err;
    kern<<<grid, wpb * 32, smem, st>>>(net, ch, s, rb);
    return cudaGetLastError();
}

// Finish of a screened step (after the propose kernel and the layer-2 GEMM),
// two chains per warp: chain 2w + h's chosen moves s = 0, 1 (at most two) are
// simulated together in byte lane 2h + s, whose tables are the chain's x_cur
// with that one move applied (Table 1's Simulate of x with one parameter
// changed); then for each chain the move of lowest exact score (first on ties)
// goes to the Metropolis test and commit of screen_accept.  A step without a
// candidate is a null move.  The scores are the exact ones of the one-chain
// finish, which simulates the moves one after the other.
template <int NPL, int D0, int D1>
__global__ void __launch_bounds__(kScreenWarps * 32)
    screen_finish_c4_kernel(ScreenArgs a, DevSched sc)
{
    extern __shared__ __align__(256) uint8_t sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c0 = 2 * (blockIdx.x * kScreenWarps + warp);
    if (c0 >= a.ch.n) return;
    const int nc = min(2, a.ch.n - c0);   // a lone last chain fills both halves
    const DevNet &net = a.net;
    uint4 r[2];
    int chosen[2][kMaxTop];
    int8_t *x[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int c = c0 + min(h, nc - 1);
        r[h] = step_draw(a.ch, a.g, c, 0u);
        select_candidates(a, c, lane, r[h], chosen[h]);
        x[h] = a.ch.x_cur + (size_t)c * a.ch.pstride;
    }
    if (chosen[0][0] < 0 && chosen[1][0] < 0) {
        if (lane == 0)
            for (int h = 0; h < nc; ++h) a.ch.cnt[3 * (size_t)(c0 + h) + 2] += 1;
        return;
    }
    Regs4<NPL, D0, D1> R;
    Undo4 U;
    int8_t *const xs[4] = {x[0], x[0], x[1], x[1]};
    load_regs4<NPL, D0, D1>(R, net, xs, lane);
#pragma unroll
    for (int vc = 0; vc < 4; ++vc) {
        const int move = chosen[vc >> 1][vc & 1];
        if (move >= 0)
            change4<NPL, D0, D1>(R, U, net, x[vc >> 1], vc, lane, move >> 8, (int8_t)(move & 255));
    }
    __syncwarp();
    int32_t y[4];
    simulate4<NPL, D0, D1>(R, net, sm, (uint32_t)warp * kCodeBytesPerWarp, lane, y);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (h >= nc) break;
        const int c = c0 + h;
        if (chosen[h][0] < 0) {
            if (lane == 0) a.ch.cnt[3 * (size_t)c + 2] += 1;
            continue;
        }
        int best = chosen[h][0];
        int32_t d = y[2 * h];
        if (chosen[h][1] >= 0 && y[2 * h + 1] < d) {
            best = chosen[h][1];
            d = y[2 * h + 1];
        }
        screen_accept(a, sc, c, lane, r[h], best, d);
    }
}

template <int NPL, int D0, int D1>
cudaError_t finish_t(const ScreenArgs &a, const DevSched &sc, cudaStream_t st)
{
    const int warps = (a.ch.n + 1) / 2;
    const int blocks = (warps + kScreenWarps - 1) / kScreenWarps;
    screen_finish_c4_kernel<NPL, D0, D1>
        <<<blocks, kScreenWarps * 32, kScreenWarps * (size_t)kCodeBytesPerWarp, st>>>(a, sc);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_finish_chains4(const ScreenArgs &a, const DevSched &sc, int d0, int d1,
                                  cudaStream_t st)
{
    const DevNet &net = a.net;
    if (!chains4_layout(net, d0, d1) || a.top > 2) return cudaErrorNotSupported;
    if (a.ch.n <= 0) return cudaSuccess;
    if (net.npl == 1) {
        if (d0 == 4) return finish_t<1, 4, 1>(a, sc, st);
        if (d0 == 8) return finish_t<1, 8, 1>(a, sc, st);
        if (d0 == 12) return finish_t<1, 12, 1>(a, sc, st);
        return finish_t<1, 16, 1>(a, sc, st);
    }
    if (d0 == 4) return finish_t<2, 4, 4>(a, sc, st);
    if (d1 == 4) return finish_t<2, 8, 4>(a, sc, st);
    return finish_t<2, 8, 8>(a, sc, st);
}

bool chains4_layout(const DevNet &net, int d0, int d1)
{
    if (net.lanes != 32 || net.cg != 1 || net.C != 1 || net.async) return false;
    // the layouts whose four register tables fit the register budget (4 nodes
    // per lane keep the one-chain scalar update)
    if (net.npl == 1) return d0 == 4 || d0 == 8 || d0 == 12 || d0 == 16;
    return net.npl == 2 && ((d0 == 4 && d1 == 4) || (d0 == 8 && d1 == 4) || (d0 == 8 && d1 == 8));
}

cudaError_t launch_anneal_chains4(const DevNet &net, int d0, int d1, const DevChains &ch,
                                  const DevSched &sc, int sm_count, cudaStream_t st)
{
    if (!chains4_layout(net, d0, d1)) return cudaErrorNotSupported;
    if (ch.n <= 0 || sc.g1 <= sc.g0) return cudaSuccess;
    if (net.npl == 1) {
        if (d0 == 4) return launch_t<1, 4, 1>(net, ch, sc, sm_count, st);
        if (d0 == 8) return launch_t<1, 8, 1>(net, ch, sc, sm_count, st);
        if (d0 == 12) return launch_t<1, 12, 1>(net, ch, sc, sm_count, st);
        return launch_t<1, 16, 1>(net, ch, sc, sm_count, st);
    }
    if (d0 == 4) return launch_t<2, 4, 4>(net, ch, sc, sm_count, st);
    if (d1 == 4) return launch_t<2, 8, 4>(net, ch, sc, sm_count, st);
    return launch_t<2, 8, 8>(net, ch, sc, sm_count, st);
}

}  // namespace rn
