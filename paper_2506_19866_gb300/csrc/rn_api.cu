// rn_api.cu -- host side of the C ABI declared in include/rnanneal.h.
//
// Builds the device layout of each network (lane/slot placement of nodes,
// padded per-slot in-edge tables, error tables of the time courses), owns the
// chain state, computes the Metropolis threshold tables in double precision on
// the host (Table 1: A = exp(-dE / T)), and launches the kernels of
// rn_kernels.cu on the context stream.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <numeric>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/rnanneal.h"
#include "rn_launch.h"

#include "rn_context.h"

namespace rn {

thread_local std::string g_create_error;

int fail(rn_ctx *ctx, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    else g_create_error = buf;
    return code;
}

int cuda_fail(rn_ctx *ctx, cudaError_t e, const char *what)
{
    // The runtime also records the error for the next cudaGetLastError, which the
    // launchers check after every launch; reported here, it is cleared, so that a
    // recoverable failure (an allocation too large) does not fail a later call.
    (void)cudaGetLastError();
    return fail(ctx, e == cudaErrorMemoryAllocation ? RN_ENOMEM : RN_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

Network *get_net(rn_ctx *ctx, int32_t id)
{
    if (!ctx || id < 0 || id >= (int32_t)ctx->nets.size()) return nullptr;
    return ctx->nets[(size_t)id].get();
}

// Domain of parameter j (Sections 2.1 and 2.2).
int domain_of(const Network &n, int32_t j, int8_t vals[6])
{
    const int32_t E = n.E, N = n.N;
    if (j < E || (j >= 3 * E + N && j < 3 * E + 2 * N)) {   // w, m
        vals[0] = 0; vals[1] = 1; vals[2] = 2;
        return 3;
    }
    if (j < 2 * E) { vals[0] = -1; vals[1] = 0; vals[2] = 1; return 3; }   // p
    if (j < 3 * E || j >= 3 * E + 2 * N) { vals[0] = 1; vals[1] = 2; return 2; }   // t, d
    if (n.fast[(size_t)(j - 3 * E)]) { vals[0] = 10; vals[1] = 11; vals[2] = 12; return 3; }
    for (int k = 0; k < 6; ++k) vals[k] = (int8_t)(k + 1);
    return 6;
}

bool in_domain(const Network &n, int32_t j, int8_t v)
{
    int8_t vals[6];
    const int k = domain_of(n, j, vals);
    for (int a = 0; a < k; ++a)
        if (vals[a] == v) return true;
    return false;
}

// Domains, fixed values, and the two constraints of Section 2.5.3.
int check_vector(rn_ctx *ctx, const Network &n, const int8_t *x, int64_t which)
{
    for (int32_t j = 0; j < n.P; ++j) {
        if (!in_domain(n, j, x[j]))
            return fail(ctx, RN_EINVAL, "vector %lld: parameter %d = %d is outside its domain",
                        (long long)which, j, (int)x[j]);
        if (n.has_frozen && n.frozen[(size_t)j] && x[j] != n.frozen_val[(size_t)j])
            return fail(ctx, RN_EINVAL, "vector %lld: fixed parameter %d changed",
                        (long long)which, j);
    }
    std::vector<int> out_nz((size_t)n.N, 0), pos_in((size_t)n.N, 0);
    for (int32_t e = 0; e < n.E; ++e) {
        if (x[e] != 0) out_nz[(size_t)n.src[(size_t)e]]++;
        if (x[e] != 0 && x[n.E + e] == 1) pos_in[(size_t)n.dst[(size_t)e]]++;
    }
    for (int32_t i = 0; i < n.N; ++i)
        if (out_nz[(size_t)i] == 0 || pos_in[(size_t)i] == 0)
            return fail(ctx, RN_ECONSTRAINT,
                        "vector %lld: node %d lacks a nonzero out-edge or an activating in-edge",
                        (long long)which, i);
    return RN_OK;
}

// Acceptance threshold of Table 1 as a 32-bit word: floor(exp(-dE / T) * 2^32),
// capped at 2^32 - 1.
uint32_t threshold(double T, int64_t dE)
{
    const double a = std::exp(-(double)dE / T) * 4294967296.0;
    const double f = std::floor(a);
    return f >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)f;
}

// Parameters GetCandidate may pick (Table 1): every one that is not fixed,
// less the speeds u when the update scheme has no priorities (synchronous or
// asynchronous updating, Section 2.2), where u has no effect.
void build_free_list(Network &n)
{
    const int32_t E = n.E, N = n.N;
    n.free_list.clear();
    for (int32_t j = 0; j < n.P; ++j)
        if (!(n.has_frozen && n.frozen[(size_t)j]) &&
            !((n.sync || n.async_) && j >= 3 * E && j < 3 * E + N))
            n.free_list.push_back(j);
}

// Table rows of the block path's register variant, which keeps two copies of
// the state codes (code_word2).  For each slot and warp, row d of the table is
// read by the warp's 32 threads at once, each gathering the code of one
// source; a bank serves one 4-byte word per wavefront.  Every entry may read
// its source from either copy, which puts it in one of two banks.  Row by row,
// lanes are matched to distinct banks (augmenting paths over every remaining
// in-edge in both copies), lanes that must place an edge in this row (as many
// edges left as rows) first; a lane that must place one and found no free bank
// takes the option that adds the fewest words to a bank, and a lane with
// nothing to place reads a word the row already reads.  The image sums the
// same edges in any order, so the placement changes no result.
void place_rows_two_copies(Network &n, const std::vector<int> &dw, int W)
{
    const int L = n.lanes, npl = n.npl;
    const uint32_t copy2_word = block_code_bytes(npl) / 4u;   // word index of the second copy
    struct Opt {
        int bank, word, t;
        bool c2;
    };
    for (int slot = 0; slot < npl; ++slot)
    for (int wg = 0; wg < W; ++wg) {
        std::vector<std::vector<std::pair<int, int32_t>>> rem(32);   // (first-copy word, edge)
        for (int lane = 0; lane < 32; ++lane) {
            const int i = n.q_node[(size_t)((32 * wg + lane) * npl + slot)];
            if (i < 0) continue;
            for (int32_t k = n.in_ptr[(size_t)i]; k < n.in_ptr[(size_t)i + 1]; ++k) {
                const int32_t e = n.in_edges[(size_t)k];
                rem[(size_t)lane].push_back({n.node_q[(size_t)n.src[(size_t)e]] >> 1, e});
            }
        }
        const int rows = dw[(size_t)slot * W + wg];
        for (int d = 0; d < rows; ++d) {
            std::vector<std::vector<Opt>> opts(32);
            bool must[32];
            for (int lane = 0; lane < 32; ++lane) {
                const auto &r = rem[(size_t)lane];
                must[lane] = !r.empty() && (int)r.size() >= rows - d;
                for (int t = 0; t < (int)r.size(); ++t) {
                    const int w1 = r[(size_t)t].first;
                    const int w2 = (int)(copy2_word + code_word2((uint32_t)w1));
                    opts[(size_t)lane].push_back({w1 & 31, w1, t, false});
                    opts[(size_t)lane].push_back({w2 & 31, w2, t, true});
                }
            }
            int owner[32], choice[32];
            for (int b = 0; b < 32; ++b) owner[b] = -1;
            for (int l = 0; l < 32; ++l) choice[l] = -1;
            bool seen[32];
            // Kuhn's augmenting path from lane l over banks not yet visited
            auto augment = [&](auto &&self, int l) -> bool {
                const auto &o = opts[(size_t)l];
                for (int k = 0; k < (int)o.size(); ++k) {
                    const int b = o[(size_t)k].bank;
                    if (seen[b]) continue;
                    seen[b] = true;
                    if (owner[b] < 0 || self(self, owner[b])) {
                        owner[b] = l;
                        choice[l] = k;
                        return true;
                    }
                }
                return false;
            };
            std::vector<int> lanes(32);
            std::iota(lanes.begin(), lanes.end(), 0);
            std::stable_sort(lanes.begin(), lanes.end(), [&](int a, int b) {
                if (must[a] != must[b]) return must[a];
                return rem[(size_t)a].size() > rem[(size_t)b].size();
            });
            for (int l : lanes) {
                if (opts[(size_t)l].empty()) continue;
                for (int b = 0; b < 32; ++b) seen[b] = false;
                augment(augment, l);
            }
            std::vector<int> words[32];   // distinct words read per bank in this row
            auto note = [&](const Opt &o) {
                auto &v = words[o.bank];
                if (std::find(v.begin(), v.end(), o.word) == v.end()) v.push_back(o.word);
            };
            for (int l = 0; l < 32; ++l)
                if (choice[l] >= 0) note(opts[(size_t)l][(size_t)choice[l]]);
            for (int l = 0; l < 32; ++l) {
                if (choice[l] >= 0 || !must[l]) continue;
                int best = 0, best_cost = 1 << 30;
                for (int k = 0; k < (int)opts[(size_t)l].size(); ++k) {
                    const Opt &o = opts[(size_t)l][(size_t)k];
                    const auto &v = words[o.bank];
                    const int cost = std::find(v.begin(), v.end(), o.word) != v.end()
                                         ? 0
                                         : (int)v.size() + 1;
                    if (cost < best_cost) {
                        best_cost = cost;
                        best = k;
                    }
                }
                choice[l] = best;
                note(opts[(size_t)l][(size_t)best]);
            }
            int pad_word = 0;
            for (int b = 0; b < 32; ++b)
                if (!words[b].empty()) {
                    pad_word = words[b][0];
                    break;
                }
            for (int l = 0; l < 32; ++l) {
                const size_t at = ((size_t)slot * n.dtab + d) * L + 32 * wg + l;
                if (choice[l] < 0) {   // padding: -1 - (byte offset of a word the row reads)
                    n.edge_id[at] = -1 - 4 * pad_word;
                    continue;
                }
                const Opt &o = opts[(size_t)l][(size_t)choice[l]];
                auto &r = rem[(size_t)l];
                const int32_t e = r[(size_t)o.t].second;
                r.erase(r.begin() + o.t);
                n.edge_id[at] = e | (o.c2 ? kCodeCopy2 : 0);
                n.edge_pos[(size_t)e] = ((32 * wg + l) << 16) | (slot << 8) | d;
            }
        }
    }
}

// Node placement: nodes ranked by in-degree (descending, then index); rank r
// goes to slot r / 32, lane r % 32, internal index q = lane * npl + slot.
void build_layout(Network &n)
{
    const int32_t N = n.N, E = n.E;
    // A chain is simulated by L = 32 lanes (one warp) up to 512 nodes: 1, 2 or
    // 4 nodes per lane for the register-table kernels, ceil(N / 32) above 128
    // nodes for the shared-memory path.  Above 512 nodes a block of L = 256
    // threads holds the chain (block path), ceil(N / 256) nodes per thread
    // (rounded up to an even number below 8), up to 4096 nodes.
    // (the block path also takes networks of any size up to 4096 whose
    // in-degree exceeds the warp paths' 16; it keeps at least 2 nodes per
    // thread so that its padding rows can read the code of node 2 t)
    std::vector<int32_t> indeg((size_t)N, 0);
    for (int32_t e = 0; e < E; ++e) indeg[(size_t)n.dst[(size_t)e]]++;
    const int32_t max_in = N ? *std::max_element(indeg.begin(), indeg.end()) : 0;
    const int L = N <= 32 * kMaxSlots && max_in <= 16 ? 32 : kBlockLanes;
    n.lanes = L;
    if (L == 32)
        n.npl = N <= 32 ? 1 : N <= 64 ? 2 : N <= 128 ? 4 : (N + 31) / 32;
    else
        n.npl = N <= L * kMaxSlots ? std::max(2, (N + L - 1) / L) : 0;
    // up to 2048 nodes the block path keeps node state in registers, compiled
    // for an even number of nodes per thread
    if (L != 32 && n.npl > 0 && n.npl < 8) n.npl += n.npl & 1;
    // 129 .. 320 nodes: 6, 8 or 10 per lane, the hybrid path's compiled layouts
    if (L == 32 && N > 128 && N <= 320) n.npl = N <= 192 ? 6 : N <= 256 ? 8 : 10;
    n.in_ptr.assign((size_t)N + 1, 0);
    n.out_ptr.assign((size_t)N + 1, 0);
    for (int32_t e = 0; e < E; ++e) {
        n.in_ptr[(size_t)n.dst[(size_t)e] + 1]++;
        n.out_ptr[(size_t)n.src[(size_t)e] + 1]++;
    }
    for (int32_t i = 0; i < N; ++i) {
        n.in_ptr[(size_t)i + 1] += n.in_ptr[(size_t)i];
        n.out_ptr[(size_t)i + 1] += n.out_ptr[(size_t)i];
    }
    n.in_edges.assign((size_t)E, 0);
    n.out_edges.assign((size_t)E, 0);
    {
        std::vector<int32_t> fi(n.in_ptr.begin(), n.in_ptr.end() - 1);
        std::vector<int32_t> fo(n.out_ptr.begin(), n.out_ptr.end() - 1);
        for (int32_t e = 0; e < E; ++e) {
            n.in_edges[(size_t)fi[(size_t)n.dst[(size_t)e]]++] = e;
            n.out_edges[(size_t)fo[(size_t)n.src[(size_t)e]]++] = e;
        }
    }
    build_free_list(n);

    n.supported = false;
    if (n.npl == 0) return;
    const int npl = n.npl;
    std::vector<int32_t> order((size_t)N);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return n.in_ptr[(size_t)a + 1] - n.in_ptr[(size_t)a] >
               n.in_ptr[(size_t)b + 1] - n.in_ptr[(size_t)b];
    });
    n.node_q.assign((size_t)N, 0);
    n.q_node.assign((size_t)L * npl, (int16_t)-1);
    for (int k = 0; k < kMaxSlots; ++k) n.D[k] = 0;
    for (int32_t r = 0; r < N; ++r) {
        const int32_t i = order[(size_t)r];
        const int slot = r / L, lane = r % L;
        const int q = lane * npl + slot;
        n.node_q[(size_t)i] = q;
        n.q_node[(size_t)q] = (int16_t)i;
        n.D[slot] = std::max(n.D[slot], n.in_ptr[(size_t)i + 1] - n.in_ptr[(size_t)i]);
    }
    // The hybrid and block-register paths gather two slots per loop (twice the
    // independent loads in flight): slots 2j and 2j + 1 get the same number of
    // table rows, the extra ones neutral padding.
    const bool paired = (L == 32 && smemreg_layout(npl)) || (L != 32 && npl <= 8);
    if (paired)
        for (int k = 0; k + 1 < npl; k += 2) n.D[k] = n.D[k + 1] = std::max(n.D[k], n.D[k + 1]);
    // The block path's loop over a slot's rows needs a bound that is uniform
    // over a warp, not over the block: each warp's edges of a slot are placed
    // in the first rows, as many as the largest in-degree among its own lanes
    // (paired slots again equal), and the warp gathers only those.  Nodes are
    // ranked by in-degree, so later warps of a slot stop earlier.
    const int W = L / 32;
    std::vector<int> dw;
    n.warp_d4.clear();
    if (L != 32) {
        dw.assign((size_t)npl * W, 0);
        for (int32_t r = 0; r < N; ++r) {
            const int32_t i = order[(size_t)r];
            int &d = dw[(size_t)(r / L) * W + (r % L) / 32];
            d = std::max(d, n.in_ptr[(size_t)i + 1] - n.in_ptr[(size_t)i]);
        }
        if (paired)
            for (int k = 0; k + 1 < npl; k += 2)
                for (int wg = 0; wg < W; ++wg) {
                    int &a = dw[(size_t)k * W + wg], &b = dw[(size_t)(k + 1) * W + wg];
                    a = b = std::max(a, b);
                }
        n.warp_d4.resize(dw.size());
        for (size_t k = 0; k < dw.size(); ++k) n.warp_d4[k] = (uint8_t)((dw[k] + 3) & ~3);
    }
    n.dtab = 1;
    for (int k = 0; k < npl; ++k) n.dtab = std::max(n.dtab, n.D[k]);
    // in-degree capacity: 16 in registers (warp paths), 31 on the block path.
    // The byte-SIMD image holds 127 + K_i in one byte per condition, exact for
    // |K_i| <= 127; each edge adds at most 4 in magnitude (Section 2.1:
    // (s // t) w p with s, w <= 2), so 31 in-edges are the most a byte holds.
    if (n.dtab > (L == 32 ? 16 : 31)) return;
    // the block path's shared memory must fit one block (227 KiB on sm_103)
    if (L != 32 && block_path_smem_bytes(n.D, npl, N) > kBlockSmemMax) return;
    n.edge_id.assign((size_t)npl * n.dtab * L, -1);
    n.edge_q2.assign((size_t)E, 0);
    n.edge_pos.assign((size_t)E, 0);
    if (npl <= kRegSlots)   // one-byte code offsets of the register-table words
        for (int32_t e = 0; e < E; ++e)
            n.edge_q2[(size_t)e] = (uint8_t)(2 * n.node_q[(size_t)n.src[(size_t)e]]);
    // Column d of slot k is read by the 32 lanes of a warp at once: each lane
    // gathers the 2-byte state code of one source.  A shared-memory bank serves
    // one 4-byte word per wavefront, so the in-edges of each lane are spread over
    // the columns greedily such that no two lanes of a warp read different words
    // of one bank in a column; a padding entry reads a word already read in its
    // column.  (The block path does this for each of its 8 warps; its register
    // variant, which keeps two copies of the codes, matches lanes to banks
    // instead: place_rows_two_copies.)
    if (L != 32 && block_path_two_copies(n.D, npl, N)) {
        place_rows_two_copies(n, dw, W);
        n.supported = true;
        return;
    }
    for (int slot = 0; slot < npl; ++slot)
    for (int wg = 0; wg < L / 32; ++wg) {
        std::vector<std::vector<std::pair<int, int32_t>>> rem(32);   // (word, edge)
        for (int lane = 0; lane < 32; ++lane) {
            const int i = n.q_node[(size_t)((32 * wg + lane) * npl + slot)];
            if (i < 0) continue;
            for (int32_t k = n.in_ptr[(size_t)i]; k < n.in_ptr[(size_t)i + 1]; ++k) {
                const int32_t e = n.in_edges[(size_t)k];
                rem[(size_t)lane].push_back({n.node_q[(size_t)n.src[(size_t)e]] >> 1, e});
            }
        }
        const int rows = L == 32 ? n.D[slot] : dw[(size_t)slot * W + wg];
        for (int d = 0; d < rows; ++d) {
            int used[32];
            for (int b = 0; b < 32; ++b) used[b] = -1;
            std::vector<int> lanes(32);
            std::iota(lanes.begin(), lanes.end(), 0);
            std::stable_sort(lanes.begin(), lanes.end(), [&](int a, int b) {
                return rem[(size_t)a].size() > rem[(size_t)b].size();
            });
            std::vector<int> padded;
            for (int lane : lanes) {
                auto &r = rem[(size_t)lane];
                int pick = -1;
                for (size_t t = 0; t < r.size(); ++t) {
                    const int b = r[t].first & 31;
                    if (used[b] < 0 || used[b] == r[t].first) {
                        pick = (int)t;
                        break;
                    }
                }
                if (pick < 0 && !r.empty() && (int)r.size() >= rows - d) pick = 0;
                if (pick < 0) {
                    padded.push_back(lane);
                    continue;
                }
                const int word = r[(size_t)pick].first;
                const int32_t e = r[(size_t)pick].second;
                r.erase(r.begin() + pick);
                if (used[word & 31] < 0) used[word & 31] = word;
                n.edge_id[((size_t)slot * n.dtab + d) * L + 32 * wg + lane] = e;
                n.edge_pos[(size_t)e] = ((32 * wg + lane) << 16) | (slot << 8) | d;
            }
            int pad_word = 0;
            for (int b = 0; b < 32; ++b)
                if (used[b] >= 0) {
                    pad_word = used[b];
                    break;
                }
            for (int lane : padded)   // padding: -1 - (byte offset of a read code)
                n.edge_id[((size_t)slot * n.dtab + d) * L + 32 * wg + lane] = -1 - 4 * pad_word;
        }
    }
    n.supported = true;
}

// After a synchronisation: a kernel whose bounded wait gave up has set the
// device flag; report it (and clear it) as RN_ETIMEOUT.
int check_device_flag(rn_ctx *ctx)
{
    int32_t flag = 0;
    RN_CUDA(ctx, cudaMemcpy(&flag, ctx->dev_err.p, sizeof flag, cudaMemcpyDeviceToHost));
    if (!flag) return RN_OK;
    RN_CUDA(ctx, cudaMemset(ctx->dev_err.p, 0, sizeof flag));
    return fail(ctx, RN_ETIMEOUT,
                "a bounded device-side wait gave up (code %d: 1 = anneal work item, 2 = "
                "tensor-core pipeline); results of the calls since the last check are "
                "incomplete",
                flag);
}

int require_supported(rn_ctx *ctx, const Network &n)
{
    if (!n.supported)
        return fail(ctx, RN_EUNSUPPORTED,
                    "network with %d nodes and maximum in-degree %d is outside the compiled "
                    "kernels (N <= 512 with in-degree <= 16, or N <= 4096 with in-degree <= 31)",
                    n.N, n.dtab);
    return RN_OK;
}

int evaluate_device_impl(rn_ctx *ctx, Network &n, int32_t count, const int8_t *x, int64_t xstride,
                         int32_t *score, int32_t *score2, uint8_t *traj)
{
    if (count <= 0) return RN_OK;
    const cudaError_t e = launch_evaluate(n.dev(), x, xstride, count, score, score2, traj,
                                          ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "evaluate kernel");
    ctx->launches += 1;
    return RN_OK;
}

int alloc_chains(rn_ctx *ctx, Network &n, int32_t count)
{
    n.pstride = (n.P + 15) & ~15;
    const size_t rows = (size_t)count * (size_t)n.pstride;
    RN_CUDA(ctx, n.d_x_cur.reserve(rows));
    RN_CUDA(ctx, n.d_x_best.reserve(rows));
    RN_CUDA(ctx, n.d_d_cur.reserve((size_t)count));
    RN_CUDA(ctx, n.d_d_best.reserve((size_t)count));
    RN_CUDA(ctx, n.d_cnt.reserve((size_t)count * 3));
    n.n_chains = count;
    return RN_OK;
}

int upload_rows(rn_ctx *ctx, Network &n, int8_t *dst, const int8_t *src, int32_t count)
{
    std::vector<int8_t> rows((size_t)count * n.pstride, 0);
    for (int32_t c = 0; c < count; ++c)
        std::memcpy(&rows[(size_t)c * n.pstride], src + (size_t)c * n.P, (size_t)n.P);
    RN_CUDA(ctx, cudaMemcpyAsync(dst, rows.data(), rows.size(), cudaMemcpyHostToDevice,
                                 ctx->stream));
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return RN_OK;
}

int download_rows(rn_ctx *ctx, const Network &n, int8_t *dst, const int8_t *src)
{
    std::vector<int8_t> rows((size_t)n.n_chains * n.pstride);
    RN_CUDA(ctx, cudaMemcpyAsync(rows.data(), src, rows.size(), cudaMemcpyDeviceToHost,
                                 ctx->stream));
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int32_t c = 0; c < n.n_chains; ++c)
        std::memcpy(dst + (size_t)c * n.P, &rows[(size_t)c * n.pstride], (size_t)n.P);
    return RN_OK;
}

// Threshold tables of levels [l0, l1]: T_l by repeated multiplication from T0,
// D_l = the largest dE <= cap with a nonzero threshold (cap = the largest dE
// any candidate can reach, and beyond 32 ln 2 T the threshold is 0).
int build_thresholds(rn_ctx *ctx, const rn_schedule &s, int64_t l0, int64_t l1, int64_t max_dE,
                     std::vector<uint32_t> &thr, std::vector<int32_t> &off,
                     std::vector<int32_t> &len)
{
    double T = s.T0;
    for (int64_t l = 0; l < l0; ++l) T *= s.alpha;
    thr.clear();
    off.clear();
    len.clear();
    for (int64_t l = l0; l <= l1; ++l) {
        if (l > l0) T *= s.alpha;
        if (!(T > 0.0) || !std::isfinite(T))
            return fail(ctx, RN_EINVAL, "temperature of level %lld is not a positive number",
                        (long long)l);
        const double lim = std::floor(22.2 * T) + 2.0;
        const int64_t cap = std::min<int64_t>(max_dE, lim > 1e9 ? (int64_t)1e9 : (int64_t)lim);
        off.push_back((int32_t)thr.size());
        int64_t D = 0;
        const size_t start = thr.size();
        for (int64_t dE = 1; dE <= cap; ++dE) {
            const uint32_t t = threshold(T, dE);
            thr.push_back(t);
            if (t != 0) D = dE;
        }
        thr.resize(start + (size_t)D);
        len.push_back((int32_t)D);
        if (thr.size() > (size_t)1 << 30)
            return fail(ctx, RN_ENOMEM, "threshold tables exceed 2^30 entries");
    }
    return RN_OK;
}

// Threshold tables of levels [l0, l1] into sc: the schedule cache when it
// covers them (cached = true), else freshly built into the context buffers.
int thresholds_for(rn_ctx *ctx, const rn_schedule &s, int64_t l0, int64_t l1, int64_t cap,
                   DevSched &sc, bool &cached)
{
    const SchedCache &cc = ctx->cache;
    cached = cc.valid && cc.T0 == s.T0 && cc.alpha == s.alpha && cc.iters == s.iters_per_level &&
             l0 >= cc.l0 && l1 <= cc.l1 && cc.cap >= cap;
    if (cached) {
        sc.level0 = cc.l0;
        sc.thr_off = cc.off.p;
        sc.thr_len = cc.len.p;
        sc.thr = cc.thr.p;
        return RN_OK;
    }
    std::vector<uint32_t> thr;
    std::vector<int32_t> off, len;
    int rc = build_thresholds(ctx, s, l0, l1, cap, thr, off, len);
    if (rc) return rc;
    if (thr.empty()) thr.push_back(0);
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));   // earlier launches may read the tables
    RN_CUDA(ctx, ctx->thr.reserve(thr.size()));
    RN_CUDA(ctx, ctx->thr_off.reserve(off.size()));
    RN_CUDA(ctx, ctx->thr_len.reserve(len.size()));
    RN_CUDA(ctx, cudaMemcpy(ctx->thr.p, thr.data(), thr.size() * sizeof(uint32_t),
                            cudaMemcpyHostToDevice));
    RN_CUDA(ctx, cudaMemcpy(ctx->thr_off.p, off.data(), off.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice));
    RN_CUDA(ctx, cudaMemcpy(ctx->thr_len.p, len.data(), len.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice));
    sc.level0 = l0;
    sc.thr_off = ctx->thr_off.p;
    sc.thr_len = ctx->thr_len.p;
    sc.thr = ctx->thr.p;
    return RN_OK;
}

// Networks annealed together in one launch: every network with chains, when
// all of them use groups of 4 conditions (the batched kernel's update).
// A network the batched kernel takes: chains, groups of 4 conditions, and a
// warp per chain.  The others (one condition, or the block path) are annealed
// by their own launches beside the batch.
bool in_batch(const Network &n) { return n.chains_valid && n.cg == 4 && n.lanes == 32; }

bool batchable(rn_ctx *ctx, const rn_schedule &s)
{
    int k = 0;
    for (auto &np : ctx->nets) k += in_batch(*np);
    return k >= 2 && !s.global_sync;
}

// Global chain lists for the current table paths: the chains of networks on
// large regions first (shared-memory or hybrid tables: the large-region
// warps' queue), then the rest.  Each class is grouped by table path
// (descending: 8, 6, 0 and 4, 2, 1 nodes per lane, which also follows network
// size), in work order within a path, so that the warps in flight mostly run
// one path's code at a time.
int batch_items(rn_ctx *ctx, BatchState &B)
{
    std::vector<int32_t> item_net, item_chain;
    int32_t big = 0;
    std::vector<size_t> seq(B.order.size());
    std::iota(seq.begin(), seq.end(), 0);
    std::stable_sort(seq.begin(), seq.end(),
                     [&](size_t a, size_t b) { return B.host_path[a] > B.host_path[b]; });
    B.phases.clear();
    for (int pass = 0; pass < 2; ++pass)
        for (size_t b : seq) {
            if (batch_shared_tables(B.host_path[b]) != (pass == 0)) continue;
            const Network &n = *ctx->nets[(size_t)B.order[b]];
            // a phase of a phased launch: the run of global chains of one path
            const int32_t path = B.host_path[b];
            if (B.phases.empty() || B.phases.back().path != path) {
                BatchPhase ph{};
                ph.path = path;
                ph.r0 = (int32_t)item_net.size();
                ph.queue = (int32_t)B.phases.size();
                B.phases.push_back(ph);
            }
            B.phases.back().n += n.n_chains;
            for (int32_t c = 0; c < n.n_chains; ++c) {
                item_net.push_back((int32_t)b);
                item_chain.push_back(c);
            }
            if (pass == 0) big += n.n_chains;
        }
    if (B.phases.size() > (size_t)kMaxPhases)
        return fail(ctx, RN_EINVAL, "%zu table paths in one batch", B.phases.size());
    B.total = (int32_t)item_net.size();
    B.total_big = big;
    RN_CUDA(ctx, B.item_net.upload(item_net));
    RN_CUDA(ctx, B.item_chain.upload(item_chain));
    return RN_OK;
}

// Warps per block of a phased launch's phase of table path `path` (paths
// 0, 1, 2, 4, 6, 8, 10 index the slots 0 .. 6); 4 until tuned.
int phase_slot(int path)
{
    return path == 0 ? 0 : path == 1 ? 1 : path == 2 ? 2 : path == 4 ? 3 : path == 6 ? 4
         : path == 8 ? 5 : 6;
}

int phase_wpb_of(const BatchState &B, int path)
{
    const size_t k = (size_t)phase_slot(path);
    return k < B.phase_wpb.size() && B.phase_wpb[k] > 0 ? B.phase_wpb[k] : 4;
}

// Item lists, warp regions (large: any network; small: register-table
// networks), large-region warps per block (all when every network is on the
// shared-memory tables, none without such networks, otherwise their share of
// the work rounded up) and the resident grid of the current configuration.
int batch_region(rn_ctx *ctx, BatchState &B)
{
    int rc = batch_items(ctx, B);
    if (rc) return rc;
    B.region_bytes = 16;
    B.region_small = 16;
    double work_big = 0, work_all = 0;
    for (size_t b = 0; b < B.order.size(); ++b) {
        const Network &n = *ctx->nets[(size_t)B.order[b]];
        const bool big = batch_shared_tables(B.host_path[b]);
        const uint32_t r = batch_region_bytes(B.host_path[b], n.D, n.npl, n.pstride, n.N);
        B.region_bytes = std::max(B.region_bytes, r);
        if (!big) B.region_small = std::max(B.region_small, r);
        const double w = (double)n.n_chains * n.C * std::max(1, n.T - 1) * (n.N + n.E);
        work_all += w;
        if (big) work_big += w;
    }
    if (B.total_big == 0) B.large = 0;
    else if (B.total_big == B.total || B.all_large) B.large = B.wpb;
    else
        B.large = std::min(B.wpb - 1,
                           std::max(1, (int)std::ceil(B.wpb * work_big / std::max(work_all, 1.0))));
    RN_CUDA(ctx, B.path.upload(B.host_path));
    if (B.phased) {
        // each phase's warp region fits that path's largest network
        for (BatchPhase &ph : B.phases) {
            ph.region = 16;
            for (size_t b = 0; b < B.order.size(); ++b)
                if (B.host_path[b] == ph.path) {
                    const Network &n = *ctx->nets[(size_t)B.order[b]];
                    ph.region = std::max(ph.region, batch_region_bytes(ph.path, n.D, n.npl,
                                                                       n.pstride, n.N));
                }
            ph.wpb = phase_wpb_of(B, ph.path);
            const cudaError_t e = batch_phase_grid(ph, ctx->sm_count);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "batched phase configuration");
        }
        return RN_OK;
    }
    const size_t smem = batch_smem_bytes(B.wpb, B.large, B.region_bytes, B.region_small);
    const cudaError_t e = batch_resident_warps(B.wpb, smem, ctx->sm_count, &B.grid);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batched kernel configuration");
    return RN_OK;
}

// Chunks of the batched launch: always 16-step chunks when the two classes
// split the warps (a class may hold more chains than its warps), else as for
// one network.
void plan_batch_chunks(const BatchState &B, DevSched &sc)
{
    const bool split = B.large > 0 && B.large < B.wpb;
    plan_chunks(sc, B.total, split ? 1 : (int64_t)B.grid * B.wpb);
}

int upload_batch_steps(rn_ctx *ctx, BatchState &B)
{
    std::vector<int64_t> g0;
    for (int id : B.order) g0.push_back(ctx->nets[(size_t)id]->step);
    RN_CUDA(ctx, cudaMemcpyAsync(B.g0.p, g0.data(), sizeof(int64_t) * g0.size(),
                                 cudaMemcpyHostToDevice, ctx->stream));
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    B.g0_synced = true;
    return RN_OK;
}

// Descriptors of every network with chains: work order (most work per chain
// first), global chain lists, default table paths (register tables where the
// batched kernel's capacities fit, shared memory otherwise).
int build_batch(rn_ctx *ctx)
{
    BatchState &B = ctx->batch;
    B.drop_graph();
    B.valid = false;
    B.order.clear();
    for (size_t id = 0; id < ctx->nets.size(); ++id)
        if (in_batch(*ctx->nets[id])) B.order.push_back((int)id);
    auto work = [&](int id) {
        const Network &n = *ctx->nets[(size_t)id];
        return (int64_t)n.C * std::max(1, n.T - 1) * (n.N + n.E);
    };
    std::stable_sort(B.order.begin(), B.order.end(),
                     [&](int a, int b) { return work(a) > work(b); });
    std::vector<DevNet> nets;
    std::vector<DevChains> chains;
    B.host_path.clear();
    int64_t total = 0;
    for (size_t b = 0; b < B.order.size(); ++b) {
        const Network &n = *ctx->nets[(size_t)B.order[b]];
        nets.push_back(n.dev());
        chains.push_back(n.chains());
        int drest = 0;
        for (int k = 1; k < n.npl; ++k) drest = std::max(drest, n.D[k]);
        B.host_path.push_back(batch_path_fits(n.npl, n.D[0], drest) ? n.npl : 0);
        total += n.n_chains;
    }
    if (total > INT32_MAX / 2) return fail(ctx, RN_EINVAL, "too many chains in the batch");
    RN_CUDA(ctx, B.nets.upload(nets));
    RN_CUDA(ctx, B.chains.upload(chains));
    RN_CUDA(ctx, B.g0.alloc(B.order.size()));
    RN_CUDA(ctx, ctx->done.reserve((size_t)total));
    int rc = batch_region(ctx, B);
    if (rc) return rc;
    if ((rc = upload_batch_steps(ctx, B))) return rc;
    B.tuned = false;
    B.valid = true;
    B.gen = ctx->gen;
    return RN_OK;
}

DevBatch batch_desc(const BatchState &B, int64_t sweeps)
{
    DevBatch d{};
    d.n_nets = (int32_t)B.order.size();
    d.total = B.total;
    d.total_big = B.total_big;
    d.large = B.large;
    d.sweeps = sweeps;
    d.region_bytes = B.region_bytes;
    d.region_small = B.region_small;
    d.nets = B.nets.p;
    d.chains = B.chains.p;
    d.g0 = B.g0.p;
    d.item_net = B.item_net.p;
    d.item_chain = B.item_chain.p;
    d.path = B.path.p;
    return d;
}

// Autotuner.  Candidates c < 8 are single launches: c < 6 the table paths
// (c % 3: register tables where they fit and shared-memory tables elsewhere /
// the same with the hybrid path for 6 or 8 nodes per lane / shared-memory
// tables for all) x warps per block (c / 3: 4 / 2), large-region warps by the
// work share; c = 6, 7: register tables where they fit, 4 / 2 warps per block,
// every warp with a large region (no warp idles once the register-table work
// is done).  c = 8, 9 are phased launches, one kernel per table path (8: the
// paths of candidate 0, 9: those of candidate 1), each phase with the warps per
// block (4 or 2) that its own trial timed faster.  Each candidate is timed on
// the real batch for a few steps from the current state, which is saved before
// and restored after the trials; the fastest is kept.
int tune_batch(rn_ctx *ctx, const DevSched &sc0, int64_t sweeps)
{
    BatchState &B = ctx->batch;
    size_t bytes = 0;
    for (int id : B.order) {
        const Network &n = *ctx->nets[(size_t)id];
        bytes += (size_t)n.n_chains * (2 * (size_t)n.pstride + 8 + 24);
    }
    DevBuf<uint8_t> save;
    RN_CUDA(ctx, save.alloc(bytes));
    auto copy_state = [&](bool to_save) -> int {
        size_t o = 0;
        for (int id : B.order) {
            const Network &n = *ctx->nets[(size_t)id];
            const size_t rows = (size_t)n.n_chains * n.pstride;
            void *bufs[5] = {n.d_x_cur.p, n.d_x_best.p, n.d_d_cur.p, n.d_d_best.p, n.d_cnt.p};
            const size_t sz[5] = {rows, rows, 4 * (size_t)n.n_chains, 4 * (size_t)n.n_chains,
                                  24 * (size_t)n.n_chains};
            for (int k = 0; k < 5; ++k) {
                void *dst = to_save ? (void *)(save.p + o) : bufs[k];
                const void *src = to_save ? bufs[k] : (const void *)(save.p + o);
                RN_CUDA(ctx, cudaMemcpyAsync(dst, src, sz[k], cudaMemcpyDeviceToDevice,
                                             ctx->stream));
                o += sz[k];
            }
        }
        return RN_OK;
    };
    // hybrid: 6 or 8 nodes per lane in the single launch, also 10 in a phased
    // one (its phase kernel is compiled for 10 nodes' registers)
    std::vector<int32_t> best_fit(B.order.size(), 0), hybrid(B.order.size(), 0);
    std::vector<int32_t> hybrid_phased(B.order.size(), 0);
    for (size_t b = 0; b < B.order.size(); ++b) {
        const Network &n = *ctx->nets[(size_t)B.order[b]];
        int drest = 0;
        for (int k = 1; k < n.npl; ++k) drest = std::max(drest, n.D[k]);
        best_fit[b] = batch_path_fits(n.npl, n.D[0], drest) ? n.npl : 0;
        const bool h = best_fit[b] == 0 && smemreg_layout(n.npl);
        hybrid[b] = h && n.npl <= 8 ? n.npl : best_fit[b];
        hybrid_phased[b] = h ? n.npl : best_fit[b];
    }
    const std::vector<int32_t> all_smem(B.host_path.size(), 0);
    auto apply = [&](int cfg, int phase_wpb) {
        B.phased = cfg >= 8;
        B.all_large = cfg == 6 || cfg == 7;
        B.host_path = cfg >= 8 ? (cfg == 8 ? best_fit : hybrid_phased)
                      : cfg >= 6 || cfg % 3 == 0 ? best_fit
                      : cfg % 3 == 1 ? hybrid : all_smem;
        B.wpb = cfg >= 8 ? 4 : cfg >= 6 ? (cfg == 6 ? 4 : 2) : cfg / 3 == 0 ? 4 : 2;
        if (phase_wpb) B.phase_wpb.assign(kMaxPhases, phase_wpb);
        B.cfg = cfg;
    };
    if (B.force >= 0 && B.force < 8) {
        apply(B.force, 0);
        int rc = batch_region(ctx, B);
        if (rc) return rc;
        B.tuned = true;
        return RN_OK;
    }
    const int64_t trial = std::min<int64_t>(sweeps, 16);
    double best = 1e300;
    int best_cfg = 0;
    std::vector<int32_t> best_phase_wpb;
    cudaEvent_t ev[2 + 2 * kMaxPhases];
    for (auto &e : ev) RN_CUDA(ctx, cudaEventCreate(&e));
    // one trial of the current configuration; phase times into phase_ms
    auto run_trial = [&](double &ms_total, std::vector<double> &phase_ms) -> int {
        int rc = batch_region(ctx, B);
        if (rc) return rc;
        DevSched sc = sc0;
        sc.g0 = 0;
        sc.g1 = trial;
        const DevBatch d = batch_desc(B, trial);
        cudaEventRecord(ev[0], ctx->stream);
        cudaError_t e;
        if (B.phased) {
            e = launch_batch_phased(d, sc, B.phases.data(), (int)B.phases.size(), ctx->stream,
                                    ev + 2);
        } else {
            plan_batch_chunks(B, sc);
            e = launch_batch(d, sc, B.wpb, B.grid, ctx->stream);
        }
        cudaEventRecord(ev[1], ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "batched kernel (autotune)");
        if (cudaEventSynchronize(ev[1]) != cudaSuccess) return RN_ECUDA;
        float ms = 0;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        ms_total = ms;
        phase_ms.assign(B.phases.size(), 0.0);
        if (B.phased)
            for (size_t k = 0; k < B.phases.size(); ++k) {
                float pm = 0;
                cudaEventElapsedTime(&pm, ev[2 + 2 * k], ev[3 + 2 * k]);
                phase_ms[k] = pm;
            }
        if ((rc = copy_state(false))) return rc;
        if ((rc = upload_batch_steps(ctx, B))) return rc;
        ctx->launches += B.phased ? (int64_t)B.phases.size() + 1 : 2;
        return RN_OK;
    };
    int rc = copy_state(true);
    for (int cfg = 0; cfg < kBatchCandidates && !rc; ++cfg) {
        if (B.force >= 0 && cfg != B.force) continue;
        if (cfg < 8) {
            apply(cfg, 0);
            double ms = 0;
            std::vector<double> pm;
            if ((rc = run_trial(ms, pm))) break;
            B.tune_ms[cfg] = ms;
            if (ms < best) { best = ms; best_cfg = cfg; }
            continue;
        }
        // phased: every phase at 4 and at 2 warps per block, each phase keeps
        // its faster one; the candidate's time is the sum of its phases'
        std::vector<double> t4, t2;
        double ms = 0;
        apply(cfg, 4);
        if ((rc = run_trial(ms, t4))) break;
        apply(cfg, 2);
        if ((rc = run_trial(ms, t2))) break;
        std::vector<int32_t> pw(kMaxPhases, 4);
        double sum = 0;
        for (size_t k = 0; k < B.phases.size(); ++k) {
            const int slot = phase_slot(B.phases[k].path);
            pw[(size_t)slot] = t2[k] < t4[k] ? 2 : 4;
            sum += std::min(t2[k], t4[k]);
        }
        B.tune_ms[cfg] = sum;
        if (sum < best) { best = sum; best_cfg = cfg; best_phase_wpb = pw; }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (rc) return rc;
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (int frc = check_device_flag(ctx)) return frc;
    apply(best_cfg, 0);
    if (best_cfg >= 8) B.phase_wpb = best_phase_wpb;
    if ((rc = batch_region(ctx, B))) return rc;
    B.tuned = true;
    return RN_OK;
}

// Every network with chains advances by `sweeps` steps in one persistent
// launch; with cached threshold tables the launch is replayed from a CUDA graph.
int anneal_batched(rn_ctx *ctx, const rn_schedule &s, int64_t sweeps)
{
    BatchState &B = ctx->batch;
    int rc;
    if (!B.valid || B.gen != ctx->gen)
        if ((rc = build_batch(ctx))) return rc;
    const int64_t iters = s.iters_per_level;
    int64_t lmin = INT64_MAX, lmax = 0, cap = 1;
    for (int id : B.order) {
        const Network &n = *ctx->nets[(size_t)id];
        lmin = std::min(lmin, n.step / iters);
        lmax = std::max(lmax, (n.step + sweeps - 1) / iters);
        cap = std::max(cap, n.max_score);
    }
    DevSched sc{};
    bool cached = false;
    if ((rc = thresholds_for(ctx, s, lmin, lmax, cap, sc, cached))) return rc;
    sc.iters = iters;
    sc.reset_to_best = s.reset_to_best;
    sc.early_reject = s.early_reject;
    sc.queue = ctx->queue.p;
    sc.done = ctx->done.p;
    sc.err = ctx->dev_err.p;
    if (!B.tuned) {
        B.drop_graph();
        if ((rc = tune_batch(ctx, sc, sweeps))) return rc;
    }
    if (!B.g0_synced) {
        B.drop_graph();
        if ((rc = upload_batch_steps(ctx, B))) return rc;
    }
    sc.g0 = 0;
    sc.g1 = sweeps;
    plan_batch_chunks(B, sc);
    const DevBatch d = batch_desc(B, sweeps);
    auto launch = [&]() {
        return B.phased ? launch_batch_phased(d, sc, B.phases.data(), (int)B.phases.size(),
                                              ctx->stream, nullptr)
                        : launch_batch(d, sc, B.wpb, B.grid, ctx->stream);
    };
    const int64_t per_call = B.phased ? (int64_t)B.phases.size() + 1 : 2;
    if (cached) {
        const bool same = B.exec && B.graph_sweeps == sweeps && B.graph_early == s.early_reject;
        if (!same) {
            B.drop_graph();
            RN_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
            const cudaError_t e = launch();
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(ctx->stream, &g);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "batched kernel (capture)");
            if (ec != cudaSuccess) return cuda_fail(ctx, ec, "cudaStreamEndCapture");
            B.graph = g;
            RN_CUDA(ctx, cudaGraphInstantiate(&B.exec, B.graph, 0));
            B.graph_sweeps = sweeps;
            B.graph_early = s.early_reject;
        }
        RN_CUDA(ctx, cudaGraphLaunch(B.exec, ctx->stream));
    } else {
        const cudaError_t e = launch();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "batched kernel");
    }
    ctx->launches += per_call;
    for (int id : B.order) ctx->nets[(size_t)id]->step += sweeps;
    return RN_OK;
}

// Message of a failed call that has no context (read with rn_last_error(NULL)).
void set_detached_error(const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_create_error = buf;
}

namespace {
PFN_cuMemGetAddressRange_v3020 address_range_fn()
{
    static PFN_cuMemGetAddressRange_v3020 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 3020, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuMemGetAddressRange_v3020>(p);
        else
            (void)cudaGetLastError();
    }
    return fn;
}
}  // namespace

// A caller's device buffer of at least `bytes` bytes from p: device memory of
// `device` (or managed memory), with [p, p + bytes) inside one allocation.
// Anything else -- a host pointer, another device's memory, a span past the
// end of its allocation -- would make a kernel fault, so it is refused here,
// before any launch.  Writes the reason to `why` and returns RN_EINVAL.
int check_device_span(const void *p, size_t bytes, int device, const char *name, char *why,
                      size_t why_len)
{
    cudaPointerAttributes a;
    const cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        snprintf(why, why_len, "%s: not a pointer the CUDA runtime knows (%s)", name,
                 cudaGetErrorString(e));
        return RN_EINVAL;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) {
        snprintf(why, why_len, "%s: host memory where device memory is required", name);
        return RN_EINVAL;
    }
    if (a.type == cudaMemoryTypeDevice && a.device != device) {
        snprintf(why, why_len, "%s: memory of device %d, the call runs on device %d", name,
                 a.device, device);
        return RN_EINVAL;
    }
    PFN_cuMemGetAddressRange_v3020 range = address_range_fn();
    CUdeviceptr base = 0;
    size_t size = 0;
    if (range && range(&base, &size, (CUdeviceptr)(uintptr_t)p) == CUDA_SUCCESS) {
        const uint64_t lo = (uint64_t)(uintptr_t)p, end = (uint64_t)base + size;
        if (lo + bytes > end) {
            snprintf(why, why_len,
                     "%s: %zu bytes needed, %llu left in its allocation from that address",
                     name, bytes, (unsigned long long)(end - lo));
            return RN_EINVAL;
        }
    }
    return RN_OK;
}
}  // namespace rn

using namespace rn;

extern "C" {

int rn_create(rn_ctx **out, int device, void *stream)
{
    if (!out) return fail(nullptr, RN_EINVAL, "out is NULL");
    *out = nullptr;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess)
        return fail(nullptr, RN_ECUDA, "cudaSetDevice(%d): %s", device, cudaGetErrorString(e));
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess)
        return fail(nullptr, RN_ECUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
    if (prop.major != 10 || prop.minor != 3)
        return fail(nullptr, RN_ECUDA, "device %d is sm_%d%d; this library is built for sm_103a",
                    device, prop.major, prop.minor);
    auto ctx = std::make_unique<rn_ctx>();
    ctx->device = device;
    ctx->sm_count = prop.multiProcessorCount;
    if (stream) {
        ctx->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess)
            return fail(nullptr, RN_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
        ctx->own_stream = true;
    }
    if (ctx->status.alloc(1) != cudaSuccess || ctx->winner.alloc(1) != cudaSuccess ||
        ctx->queue.alloc(kQueueSlots) != cudaSuccess || ctx->done.alloc(1) != cudaSuccess ||
        ctx->dev_err.alloc(1) != cudaSuccess)
        return fail(nullptr, RN_ENOMEM, "cannot allocate context buffers");
    if (cudaMemset(ctx->dev_err.p, 0, sizeof(int32_t)) != cudaSuccess)
        return fail(nullptr, RN_ECUDA, "cannot clear the device error flag");
    *out = ctx.release();
    return RN_OK;
}

int rn_destroy(rn_ctx *ctx)
{
    if (!ctx) return RN_OK;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return RN_OK;
}

const char *rn_last_error(const rn_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

int rn_load_network(rn_ctx *ctx, int32_t n_nodes, int32_t n_edges, const int32_t *src,
                    const int32_t *dst, const uint8_t *fast, const uint8_t *frozen,
                    const int8_t *frozen_val, int32_t *net_id)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    if (!src || !dst || !fast || !net_id) return fail(ctx, RN_EINVAL, "NULL array");
    if (n_nodes < 1 || n_nodes > 65535) return fail(ctx, RN_EINVAL, "n_nodes %d out of range", n_nodes);
    if (n_edges < 1) return fail(ctx, RN_EINVAL, "n_edges %d out of range", n_edges);
    if (3 * (int64_t)n_edges + 3 * (int64_t)n_nodes > INT32_MAX)
        return fail(ctx, RN_EINVAL, "P = 3E + 3N exceeds 2^31 - 1");
    if ((frozen == nullptr) != (frozen_val == nullptr))
        return fail(ctx, RN_EINVAL, "frozen and frozen_val must both be given or both be NULL");
    auto n = std::make_unique<Network>();
    n->N = n_nodes;
    n->E = n_edges;
    n->P = 3 * n_edges + 3 * n_nodes;
    n->src.assign(src, src + n_edges);
    n->dst.assign(dst, dst + n_edges);
    n->fast.assign(fast, fast + n_nodes);
    std::set<std::pair<int32_t, int32_t>> seen;
    std::vector<int> indeg((size_t)n_nodes, 0), outdeg((size_t)n_nodes, 0);
    for (int32_t e = 0; e < n_edges; ++e) {
        const int32_t a = src[e], b = dst[e];
        if (a < 0 || a >= n_nodes || b < 0 || b >= n_nodes)
            return fail(ctx, RN_EINVAL, "edge %d: node index out of range", e);
        if (a == b) return fail(ctx, RN_EINVAL, "edge %d is a self-loop", e);
        if (!seen.insert({a, b}).second) return fail(ctx, RN_EINVAL, "edge %d is a duplicate", e);
        outdeg[(size_t)a]++;
        indeg[(size_t)b]++;
    }
    for (int32_t i = 0; i < n_nodes; ++i) {
        if (fast[i] > 1) return fail(ctx, RN_EINVAL, "fast[%d] must be 0 or 1", i);
        if (indeg[(size_t)i] == 0 || outdeg[(size_t)i] == 0)
            return fail(ctx, RN_EINVAL, "node %d has no in-edge or no out-edge", i);
    }
    if (frozen) {
        n->has_frozen = true;
        n->frozen.assign(frozen, frozen + n->P);
        n->frozen_val.assign(frozen_val, frozen_val + n->P);
        for (int32_t j = 0; j < n->P; ++j) {
            if (n->frozen[(size_t)j] > 1) return fail(ctx, RN_EINVAL, "frozen[%d] must be 0 or 1", j);
            if (n->frozen[(size_t)j] && !in_domain(*n, j, n->frozen_val[(size_t)j]))
                return fail(ctx, RN_EINVAL, "fixed parameter %d is outside its domain", j);
            if (!n->frozen[(size_t)j]) n->frozen_val[(size_t)j] = 0;
        }
    } else {
        n->frozen.assign((size_t)n->P, 0);
        n->frozen_val.assign((size_t)n->P, 0);
    }
    build_layout(*n);
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    RN_CUDA(ctx, n->d_src.upload(n->src));
    RN_CUDA(ctx, n->d_dst.upload(n->dst));
    RN_CUDA(ctx, n->d_fast.upload(n->fast));
    RN_CUDA(ctx, n->d_frozen.upload(n->frozen));
    RN_CUDA(ctx, n->d_frozen_val.upload(n->frozen_val));
    RN_CUDA(ctx, n->d_free.upload(n->free_list));
    RN_CUDA(ctx, n->d_in_ptr.upload(n->in_ptr));
    RN_CUDA(ctx, n->d_in_edges.upload(n->in_edges));
    RN_CUDA(ctx, n->d_out_ptr.upload(n->out_ptr));
    RN_CUDA(ctx, n->d_out_edges.upload(n->out_edges));
    if (n->supported) {
        RN_CUDA(ctx, n->d_edge_id.upload(n->edge_id));
        RN_CUDA(ctx, n->d_edge_q2.upload(n->edge_q2));
        RN_CUDA(ctx, n->d_edge_pos.upload(n->edge_pos));
        RN_CUDA(ctx, n->d_node_q.upload(n->node_q));
        RN_CUDA(ctx, n->d_q_node.upload(n->q_node));
        if (!n->warp_d4.empty()) RN_CUDA(ctx, n->d_warp_d4.upload(n->warp_d4));
    }
    *net_id = (int32_t)ctx->nets.size();
    ctx->nets.push_back(std::move(n));
    ctx->gen++;
    return RN_OK;
}

int rn_load_timecourse(rn_ctx *ctx, int32_t net, int32_t n_cond, int32_t n_times,
                       const uint8_t *init, const uint8_t *knockout, const uint8_t *ref,
                       const uint8_t *observed)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    Network *n = get_net(ctx, net);
    if (!n) return fail(ctx, RN_EINVAL, "unknown network %d", net);
    if (!init || !ref || !observed) return fail(ctx, RN_EINVAL, "NULL array");
    if (n_cond < 1 || n_times < 1) return fail(ctx, RN_EINVAL, "n_cond and n_times must be >= 1");
    if ((int64_t)n_times > 128)
        return fail(ctx, RN_EINVAL, "n_times %d exceeds 128", n_times);
    const int32_t N = n->N, C = n_cond, T = n_times;
    if ((int64_t)C * T * N > ((int64_t)1 << 31))
        return fail(ctx, RN_EINVAL, "the time course has more than 2^31 entries");
    const size_t ctn = (size_t)C * T * N;
    for (size_t k = 0; k < (size_t)C * N; ++k) {
        if (init[k] > 2) return fail(ctx, RN_EINVAL, "init value %d outside 0..2", init[k]);
        if (knockout && knockout[k] > 1) return fail(ctx, RN_EINVAL, "knockout must be 0 or 1");
    }
    for (size_t k = 0; k < ctn; ++k) {
        if (observed[k] > 1) return fail(ctx, RN_EINVAL, "observed must be 0 or 1");
        if (observed[k] && ref[k] > 2) return fail(ctx, RN_EINVAL, "reference value outside 0..2");
    }
    // weight = observed * (|G| + 1), G from consecutive observed points (Section 2.3)
    std::vector<uint8_t> W(ctn, 0);
    int64_t max_score = 0, n_obs = 0;
    for (int32_t c = 0; c < C; ++c)
        for (int32_t t = 0; t < T; ++t)
            for (int32_t i = 0; i < N; ++i) {
                const size_t k = ((size_t)c * T + t) * N + i;
                if (!observed[k]) continue;
                int g = 0;
                if (t > 0 && observed[k - N]) g = std::abs((int)ref[k] - (int)ref[k - N]);
                W[k] = (uint8_t)(g + 1);
                max_score += 2 * W[k];
                ++n_obs;
            }
    // scores are summed in quarter units in 32 bits on the device
    if (max_score >= ((int64_t)1 << 30))
        return fail(ctx, RN_EINVAL, "maximum score %lld exceeds 2^30", (long long)max_score);
    if (n->async_) {
        // the selection table belongs to the previous time course: back to the
        // priority scheme (u proposed again) until the scheme is set again
        n->async_ = false;
        build_free_list(*n);
        RN_CUDA(ctx, n->d_free.upload(n->free_list));
    }
    n->C = C;
    n->T = T;
    n->max_score = max_score;
    n->n_obs = n_obs;
    n->has_tc = true;
    n->chains_valid = false;
    if (!n->supported) return RN_OK;
    const int npl = n->npl, L = n->lanes;
    // 4 conditions per group (byte-SIMD) unless there is a single condition;
    // the shared-memory and block paths always use groups of 4
    const int cg = (C >= 2 || npl > kRegSlots || L != 32) ? 4 : 1;
    const int G = (C + cg - 1) / cg;
    int drest = 0;
    for (int k = 1; k < npl; ++k) drest = std::max(drest, n->D[k]);
    anneal_capacity(npl, n->D[0], drest, &n->d0, &n->d1);
    // entry tables: per condition, byte b = W |b - R| for b = 0, 1, 2 (single
    // conditions, cg = 1); per group of 4 conditions, one compact word per time
    // point and node, byte c = R | W << 2 (W <= 3), [G][T][L][npl] (cg = 4)
    std::vector<uint32_t> obs((size_t)(cg == 1 ? C : G) * T * L * npl, 0u);
    // state codes: nibble c = initial state of condition g * cg + c; a node that
    // never moves in a condition (padding, knocked out, condition beyond C)
    // starts at 0 and has its bit k * cg + c set in out_bits
    std::vector<uint16_t> init_code((size_t)G * L * npl, 0), out_bits((size_t)G * L, 0);
    // the same per byte for the byte-SIMD path: initial states and "may move" bits
    std::vector<uint32_t> init_s4((size_t)G * L * npl, 0), movable((size_t)G * L * npl, 0);
    for (int g = 0; g < G; ++g)
        for (int q = 0; q < L * npl; ++q) {
            const int i = n->q_node[(size_t)q];
            const int lane = q / npl, slot = q % npl;
            for (int c = 0; c < cg; ++c) {
                const int cc = g * cg + c;
                const bool out =
                    i < 0 || cc >= C || (knockout && knockout[(size_t)cc * N + i]);
                if (out) {
                    if (slot * cg + c < 16)   // the scalar path's bits (at most 16 per lane)
                        out_bits[(size_t)g * L + lane] |= (uint16_t)(1u << (slot * cg + c));
                    continue;
                }
                const uint32_t s0 = init[(size_t)cc * N + i];
                init_code[(size_t)g * L * npl + q] |= (uint16_t)(s0 << (4 * c));
                init_s4[(size_t)g * L * npl + q] |= s0 << (8 * c);
                movable[(size_t)g * L * npl + q] |= 0x80u << (8 * c);
            }
        }
    if (cg == 1) {
        for (int32_t c = 0; c < C; ++c) {
            for (int q = 0; q < L * npl; ++q) {
                const int i = n->q_node[(size_t)q];
                const int lane = q / npl, slot = q % npl;
                if (i < 0) continue;
                for (int32_t t = 0; t < T; ++t) {
                    const size_t k = ((size_t)c * T + t) * N + i;
                    const int w = W[k], r = ref[k];
                    uint32_t word = 0;
                    if (w)
                        for (int b = 0; b < 3; ++b)
                            word |= (uint32_t)(w * std::abs(b - r)) << (8 * b);
                    obs[(((size_t)c * T + t) * L + lane) * npl + slot] = word;
                }
            }
        }
    } else {
        for (int g = 0; g < G; ++g)
            for (int32_t t = 0; t < T; ++t)
                for (int q = 0; q < L * npl; ++q) {
                    const int i = n->q_node[(size_t)q];
                    if (i < 0) continue;
                    uint32_t word = 0;
                    for (int c = 0; c < 4 && 4 * g + c < C; ++c) {
                        const size_t k = ((size_t)(4 * g + c) * T + t) * N + i;
                        if (W[k]) word |= (uint32_t)(ref[k] | W[k] << 2) << (8 * c);
                    }
                    obs[((size_t)g * T + t) * L * npl + (size_t)q] = word;
                }
    }
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    RN_CUDA(ctx, n->d_obs.upload(obs));
    RN_CUDA(ctx, n->d_init_code.upload(init_code));
    RN_CUDA(ctx, n->d_out_bits.upload(out_bits));
    RN_CUDA(ctx, n->d_init_s4.upload(init_s4));
    RN_CUDA(ctx, n->d_movable.upload(movable));
    n->movable_h = movable;
    n->cg = cg;
    ctx->gen++;
    n->G = G;
    return RN_OK;
}

int rn_set_update_scheme(rn_ctx *ctx, int32_t net, int32_t scheme, const int32_t *selected)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    Network *n = get_net(ctx, net);
    if (!n) return fail(ctx, RN_EINVAL, "unknown network %d", net);
    if (scheme < 0 || scheme > 2) return fail(ctx, RN_EINVAL, "scheme %d is not 0, 1 or 2", scheme);
    const int32_t N = n->N;
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    if (scheme == 2) {
        if (!selected) return fail(ctx, RN_EINVAL, "the asynchronous scheme needs `selected`");
        if (!n->has_tc) return fail(ctx, RN_ESTATE, "load the time course first");
        if (!n->supported) return require_supported(ctx, *n);
        const int32_t C = n->C, T = n->T, L = n->lanes, npl = n->npl, G = n->G;
        for (size_t k = 0; k < (size_t)C * T; ++k)
            if (selected[k] < -1 || selected[k] >= N)
                return fail(ctx, RN_EINVAL, "selected node %d outside -1 .. N-1", selected[k]);
        // the scalar single-condition path reads the selection itself
        RN_CUDA(ctx, n->d_async_sel.upload(std::vector<int32_t>(selected, selected + (size_t)C * T)));
        // groups of 4 conditions: per step, the static "may move" bits only at
        // the selected node
        if (n->cg == 4) {
            std::vector<uint32_t> mt((size_t)G * T * L * npl, 0u);
            for (int g = 0; g < G; ++g)
                for (int32_t t = 0; t < T; ++t)
                    for (int q = 0; q < L * npl; ++q) {
                        const int i = n->q_node[(size_t)q];
                        if (i < 0) continue;
                        uint32_t w = 0;
                        for (int c = 0; c < 4 && 4 * g + c < C; ++c)
                            if (selected[(size_t)(4 * g + c) * T + t] == i)
                                w |= n->movable_h[(size_t)g * L * npl + q] & (0xffu << (8 * c));
                        mt[((size_t)g * T + t) * L * npl + q] = w;
                    }
            RN_CUDA(ctx, n->d_movable_t.upload(mt));
        }
    }
    n->sync = scheme == 1;
    n->async_ = scheme == 2;
    build_free_list(*n);
    RN_CUDA(ctx, n->d_free.upload(n->free_list));
    n->chains_valid = false;
    ctx->gen++;
    return RN_OK;
}

int rn_n_params(rn_ctx *ctx, int32_t net, int32_t *n_params)
{
    if (!ctx) return RN_EINVAL;
    Network *n = get_net(ctx, net);
    if (!n || !n_params) return fail(ctx, RN_EINVAL, "unknown network %d", net);
    *n_params = n->P;
    return RN_OK;
}

int rn_init_chains(rn_ctx *ctx, int32_t net, int32_t n_chains, uint64_t seed, const int8_t *x0)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    Network *n = get_net(ctx, net);
    if (!n) return fail(ctx, RN_EINVAL, "unknown network %d", net);
    if (!n->has_tc) return fail(ctx, RN_ESTATE, "network %d has no time course", net);
    if (n_chains < 1) return fail(ctx, RN_EINVAL, "n_chains must be >= 1");
    int rc = require_supported(ctx, *n);
    if (rc) return rc;
    if (x0)
        for (int32_t c = 0; c < n_chains; ++c)
            if ((rc = check_vector(ctx, *n, x0 + (size_t)c * n->P, c))) return rc;
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    n->chains_valid = false;
    if ((rc = alloc_chains(ctx, *n, n_chains))) return rc;
    n->seed = seed;
    n->step = 0;
    const DevChains ch = n->chains();
    if (x0) {
        if ((rc = upload_rows(ctx, *n, ch.x_cur, x0, n_chains))) return rc;
        RN_CUDA(ctx, cudaMemcpyAsync(ch.x_best, ch.x_cur, (size_t)n_chains * n->pstride,
                                     cudaMemcpyDeviceToDevice, ctx->stream));
        RN_CUDA(ctx, cudaMemsetAsync(ch.cnt, 0, sizeof(int64_t) * 3 * (size_t)n_chains,
                                     ctx->stream));
    } else {
        RN_CUDA(ctx, ctx->status.reserve((size_t)n_chains));
        RN_CUDA(ctx, launch_init(n->dev(), ch, ctx->status.p, ctx->stream));
        ctx->launches += 1;
        std::vector<int32_t> st((size_t)n_chains);
        RN_CUDA(ctx, cudaMemcpyAsync(st.data(), ctx->status.p, sizeof(int32_t) * st.size(),
                                     cudaMemcpyDeviceToHost, ctx->stream));
        RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        for (int32_t c = 0; c < n_chains; ++c)
            if (st[(size_t)c] != 0)
                return fail(ctx, RN_ECONSTRAINT,
                            "chain %d: the fixed parameters leave a node without a possible "
                            "activating in-edge or nonzero out-edge", c);
    }
    if ((rc = evaluate_device_impl(ctx, *n, n_chains, ch.x_cur, n->pstride, ch.d_cur, ch.d_best,
                                   nullptr)))
        return rc;
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    n->chains_valid = true;
    ctx->gen++;
    return RN_OK;
}

namespace {

// Work of one network's chains for one sweep (the order of the side launches).
int64_t network_work(const Network &n)
{
    return (int64_t)n.n_chains * n.C * std::max(1, n.T - 1) * (n.N + n.E);
}

bool cache_covers(const SchedCache &cc, const rn_schedule &s, int64_t l0, int64_t l1, int64_t cap)
{
    return cc.valid && cc.T0 == s.T0 && cc.alpha == s.alpha && cc.iters == s.iters_per_level &&
           l0 >= cc.l0 && l1 <= cc.l1 && cc.cap >= cap;
}

// One network outside the batch advances by `sweeps` steps: one launch per
// segment on `st`, with the work-item counter `queue` and the n_chains chunk
// counters `done` of its own.  A segment ends at a level end when levels end
// with a sync, and where uncached threshold tables would exceed their budget
// (uncached tables are only built for launches on the context's stream).
int anneal_separate(rn_ctx *ctx, Network &n, const rn_schedule &s, int64_t sweeps,
                    unsigned int *queue, int32_t *done, cudaStream_t st)
{
    const int64_t iters = s.iters_per_level;
    // at most this many threshold entries per launch segment
    const size_t budget = (size_t)1 << 24;
    const DevNet dn = n.dev();
    const DevChains ch = n.chains();
    int64_t g = n.step;
    const int64_t g_end = n.step + sweeps;
    while (g < g_end) {
        int64_t seg_end = g_end;
        if (s.global_sync) seg_end = std::min(seg_end, (g / iters + 1) * iters);
        int64_t l0 = g / iters, l1 = (seg_end - 1) / iters;
        DevSched sc{};
        const SchedCache &cc = ctx->cache;
        if (cache_covers(cc, s, l0, l1, n.max_score)) {
            sc.level0 = cc.l0;
            sc.thr_off = cc.off.p;
            sc.thr_len = cc.len.p;
            sc.thr = cc.thr.p;
        } else {
            if (st != ctx->stream) return fail(ctx, RN_ESTATE, "uncached tables on a side stream");
            std::vector<uint32_t> thr;
            std::vector<int32_t> off, len;
            int rc = build_thresholds(ctx, s, l0, l1, n.max_score, thr, off, len);
            if (rc) return rc;
            while (thr.size() > budget && l1 > l0) {
                l1 = l0 + (l1 - l0) / 2;
                seg_end = std::min(seg_end, (l1 + 1) * iters);
                if ((rc = build_thresholds(ctx, s, l0, l1, n.max_score, thr, off, len))) return rc;
            }
            if (thr.empty()) thr.push_back(0);
            // the device tables may still be read by an earlier launch
            RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            RN_CUDA(ctx, ctx->thr.reserve(thr.size()));
            RN_CUDA(ctx, ctx->thr_off.reserve(off.size()));
            RN_CUDA(ctx, ctx->thr_len.reserve(len.size()));
            RN_CUDA(ctx, cudaMemcpy(ctx->thr.p, thr.data(), thr.size() * sizeof(uint32_t),
                                    cudaMemcpyHostToDevice));
            RN_CUDA(ctx, cudaMemcpy(ctx->thr_off.p, off.data(), off.size() * sizeof(int32_t),
                                    cudaMemcpyHostToDevice));
            RN_CUDA(ctx, cudaMemcpy(ctx->thr_len.p, len.data(), len.size() * sizeof(int32_t),
                                    cudaMemcpyHostToDevice));
            sc.level0 = l0;
            sc.thr_off = ctx->thr_off.p;
            sc.thr_len = ctx->thr_len.p;
            sc.thr = ctx->thr.p;
        }
        sc.g0 = g;
        sc.g1 = seg_end;
        sc.iters = iters;
        sc.reset_to_best = s.reset_to_best;
        sc.early_reject = s.early_reject;
        sc.queue = queue;
        sc.done = done;
        sc.err = ctx->dev_err.p;
        cudaError_t e = n.lanes != 32 ? launch_anneal_block(dn, ch, sc, ctx->sm_count, st)
                                      : launch_anneal(dn, n.d0, n.d1, ch, sc, ctx->sm_count, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "anneal kernel");
        ctx->launches += 1;
        if (s.global_sync && seg_end % iters == 0) {
            // one winner per group of sync_group chains (one group: 0)
            const int32_t G = s.sync_group > 0 ? s.sync_group : ch.n;
            RN_CUDA(ctx, ctx->winner.reserve((size_t)((ch.n + G - 1) / G)));
            e = launch_level_sync(ch, ctx->winner.p, s.sync_group, st);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "level sync kernels");
            ctx->launches += 2;
        }
        g = seg_end;
    }
    n.step = g_end;
    return RN_OK;
}

}  // namespace

int rn_anneal(rn_ctx *ctx, const rn_schedule *s, int64_t sweeps)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    if (!s) return fail(ctx, RN_EINVAL, "schedule is NULL");
    if (sweeps < 0) return fail(ctx, RN_EINVAL, "sweeps must be >= 0");
    if (s->iters_per_level < 1) return fail(ctx, RN_EINVAL, "iters_per_level must be >= 1");
    if (s->sync_group < 0) return fail(ctx, RN_EINVAL, "sync_group must be >= 0");
    if (!(s->T0 > 0.0) || !(s->alpha > 0.0) || !std::isfinite(s->T0) || !std::isfinite(s->alpha))
        return fail(ctx, RN_EINVAL, "T0 and alpha must be positive");
    bool any = false;
    for (auto &np : ctx->nets) any |= np->chains_valid;
    if (!any) return fail(ctx, RN_ESTATE, "no network has chains (call rn_init_chains)");
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    if (sweeps == 0) return RN_OK;
    // several networks: one persistent launch over all of their chains, and
    // separate launches for the networks it cannot take
    const bool batched = batchable(ctx, *s);
    if (!batched) ctx->batch.g0_synced = false;
    std::vector<Network *> sep;
    std::vector<int64_t> done_off;
    int64_t side_chains = 0;
    for (auto &np : ctx->nets)
        if (np->chains_valid && !(batched && in_batch(*np))) {
            sep.push_back(np.get());
            done_off.push_back(side_chains);
            side_chains += np->chains().n;
        }
    SideLaunch &S = ctx->side;
    if (S.queue.n < sep.size() || S.done.n < (size_t)side_chains) {
        // launches of earlier calls may still use the counters
        RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        RN_CUDA(ctx, S.queue.reserve(sep.size()));
        RN_CUDA(ctx, S.done.reserve((size_t)side_chains));
    }
    // Side streams when at least two launches can overlap and every separate
    // network reads prepared tables (one launch each, nothing synchronises).
    const int64_t iters = s->iters_per_level;
    bool concurrent = !s->global_sync && sep.size() + (batched ? 1u : 0u) >= 2;
    for (Network *n : sep)
        concurrent = concurrent && cache_covers(ctx->cache, *s, n->step / iters,
                                                (n->step + sweeps - 1) / iters, n->max_score);
    const BatchState &B = ctx->batch;
    const bool batch_steady = B.valid && B.gen == ctx->gen && B.tuned && B.g0_synced;
    // the autotuner times its trials with nothing beside them: an untuned
    // batch goes first, and the side streams wait for it
    const bool batch_first = batched && !(concurrent && batch_steady);
    if (batch_first)
        if (int rc = anneal_batched(ctx, *s, sweeps)) return rc;
    if (!concurrent) {
        for (size_t i = 0; i < sep.size(); ++i)
            if (int rc = anneal_separate(ctx, *sep[i], *s, sweeps, S.queue.p + i,
                                         S.done.p + done_off[i], ctx->stream))
                return rc;
        return RN_OK;
    }
    RN_CUDA(ctx, S.create());
    RN_CUDA(ctx, cudaEventRecord(S.fork, ctx->stream));
    // most work first, each onto the side stream with the least work so far:
    // the persistent grids that start later fill the earlier ones' tails
    std::vector<size_t> order(sep.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        return network_work(*sep[a]) > network_work(*sep[b]);
    });
    int64_t load[kSideStreams] = {};
    bool used[kSideStreams] = {};
    int rc = RN_OK;
    for (size_t i : order) {
        int k = 0;
        for (int j = 1; j < kSideStreams; ++j)
            if (load[j] < load[k]) k = j;
        if (!used[k]) {
            const cudaError_t e = cudaStreamWaitEvent(S.streams[k], S.fork, 0);
            if (e != cudaSuccess) {
                rc = cuda_fail(ctx, e, "cudaStreamWaitEvent (side stream)");
                break;
            }
            used[k] = true;
        }
        if ((rc = anneal_separate(ctx, *sep[i], *s, sweeps, S.queue.p + i, S.done.p + done_off[i],
                                  S.streams[k])))
            break;
        load[k] += network_work(*sep[i]);
    }
    if (!rc && batched && !batch_first) rc = anneal_batched(ctx, *s, sweeps);
    // every side stream joins the context's stream, after a failure too
    for (int k = 0; k < kSideStreams; ++k) {
        if (!used[k]) continue;
        cudaError_t e = cudaEventRecord(S.join[k], S.streams[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, S.join[k], 0);
        if (e != cudaSuccess) {
            cudaStreamSynchronize(S.streams[k]);
            if (!rc) rc = cuda_fail(ctx, e, "joining the side streams");
        }
    }
    return rc;
}

int rn_prepare_schedule(rn_ctx *ctx, const rn_schedule *s, int64_t total_steps)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    if (!s || total_steps < 1 || s->iters_per_level < 1)
        return fail(ctx, RN_EINVAL, "bad schedule or step count");
    if (!(s->T0 > 0.0) || !(s->alpha > 0.0) || !std::isfinite(s->T0) || !std::isfinite(s->alpha))
        return fail(ctx, RN_EINVAL, "T0 and alpha must be positive");
    int64_t cap = 1;
    for (auto &np : ctx->nets) cap = std::max(cap, np->max_score);
    const int64_t l1 = (total_steps - 1) / s->iters_per_level;
    std::vector<uint32_t> thr;
    std::vector<int32_t> off, len;
    int rc = build_thresholds(ctx, *s, 0, l1, cap, thr, off, len);
    if (rc) return rc;
    if (thr.empty()) thr.push_back(0);
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->batch.drop_graph();   // a replayed graph reads the old tables
    SchedCache &cc = ctx->cache;
    cc.valid = false;
    RN_CUDA(ctx, cc.thr.alloc(thr.size()));
    RN_CUDA(ctx, cc.off.alloc(off.size()));
    RN_CUDA(ctx, cc.len.alloc(len.size()));
    RN_CUDA(ctx, cudaMemcpy(cc.thr.p, thr.data(), thr.size() * sizeof(uint32_t),
                            cudaMemcpyHostToDevice));
    RN_CUDA(ctx, cudaMemcpy(cc.off.p, off.data(), off.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice));
    RN_CUDA(ctx, cudaMemcpy(cc.len.p, len.data(), len.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice));
    cc.T0 = s->T0;
    cc.alpha = s->alpha;
    cc.iters = s->iters_per_level;
    cc.l0 = 0;
    cc.l1 = l1;
    cc.cap = cap;
    cc.valid = true;
    return RN_OK;
}

int rn_selftest_wait(rn_ctx *ctx)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    int rc = check_device_flag(ctx);   // a failure of earlier work is reported as such
    if (rc) return rc;
    DevBuf<int32_t> buf;               // [0] the counter nothing advances, [1] the outcome
    RN_CUDA(ctx, buf.alloc(2));
    RN_CUDA(ctx, cudaMemsetAsync(buf.p, 0, 2 * sizeof(int32_t), ctx->stream));
    RN_CUDA(ctx, launch_wait_selftest(buf.p, ctx->dev_err.p, buf.p + 1, ctx->stream));
    ctx->launches += 1;
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    int32_t satisfied = 1;
    RN_CUDA(ctx, cudaMemcpy(&satisfied, buf.p + 1, sizeof satisfied, cudaMemcpyDeviceToHost));
    rc = check_device_flag(ctx);
    if (satisfied || rc != RN_ETIMEOUT)
        return fail(ctx, RN_ECUDA, "self-test: the wait on a counter nothing advances did not "
                                   "give up and report it (satisfied %d, status %d)",
                    satisfied, rc);
    return RN_ETIMEOUT;
}

int rn_launch_count(rn_ctx *ctx, int64_t *count)
{
    if (!ctx || !count) return RN_EINVAL;
    *count = ctx->launches;
    return RN_OK;
}

int rn_batch_config(rn_ctx *ctx, int32_t info[7], double trial_ms[10])
{
    if (!ctx || !info) return RN_EINVAL;
    const BatchState &B = ctx->batch;
    const bool on = B.valid && B.gen == ctx->gen;
    info[0] = on ? (int32_t)B.order.size() : 0;
    int32_t wpb = B.wpb;
    if (on && B.phased) {     // the phase with the most chains
        int32_t most = -1;
        for (const BatchPhase &ph : B.phases)
            if (ph.n > most) { most = ph.n; wpb = ph.wpb; }
    }
    info[1] = on ? wpb : 0;
    info[6] = on ? (B.phased ? (int32_t)B.phases.size() : 1) : 0;
    int32_t shared = 0, hybrid = 0;
    if (on)
        for (int32_t p : B.host_path) {
            shared += batch_shared_tables(p);
            hybrid += p > 4;
        }
    info[2] = shared;
    info[3] = on && B.exec ? 1 : 0;
    info[4] = hybrid;
    info[5] = on && B.tuned ? B.cfg : -1;
    if (trial_ms)
        for (int k = 0; k < kBatchCandidates; ++k) trial_ms[k] = B.tune_ms[k];
    return RN_OK;
}

int rn_batch_tune(rn_ctx *ctx, int32_t config)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    if (config < -1 || config >= kBatchCandidates)
        return fail(ctx, RN_EINVAL, "config %d outside -1 .. %d", config, kBatchCandidates - 1);
    ctx->batch.force = config;
    ctx->batch.tuned = false;
    ctx->batch.drop_graph();
    return RN_OK;
}

int rn_get_best(rn_ctx *ctx, int32_t net, int8_t *x, int32_t *score, int32_t *chain)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    Network *n = get_net(ctx, net);
    if (!n) return fail(ctx, RN_EINVAL, "unknown network %d", net);
    if (!n->chains_valid) return fail(ctx, RN_ESTATE, "network %d has no chains", net);
    if (!score) return fail(ctx, RN_EINVAL, "score is NULL");
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    const DevChains ch = n->chains();
    std::vector<int32_t> d((size_t)ch.n);
    RN_CUDA(ctx, cudaMemcpyAsync(d.data(), ch.d_best, sizeof(int32_t) * d.size(),
                                 cudaMemcpyDeviceToHost, ctx->stream));
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (int rc = check_device_flag(ctx)) return rc;
    int32_t b = 0;
    for (int32_t c = 1; c < ch.n; ++c)
        if (d[(size_t)c] < d[(size_t)b]) b = c;
    *score = d[(size_t)b];
    if (chain) *chain = b;
    if (x) {
        RN_CUDA(ctx, cudaMemcpyAsync(x, ch.x_best + (size_t)b * ch.pstride, (size_t)n->P,
                                     cudaMemcpyDeviceToHost, ctx->stream));
        RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return RN_OK;
}

int rn_evaluate(rn_ctx *ctx, int32_t net, int32_t count, const int8_t *x, int32_t *score,
                uint8_t *traj)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    Network *n = get_net(ctx, net);
    if (!n) return fail(ctx, RN_EINVAL, "unknown network %d", net);
    if (!n->has_tc) return fail(ctx, RN_ESTATE, "network %d has no time course", net);
    if (count < 0 || (count > 0 && (!x || !score))) return fail(ctx, RN_EINVAL, "bad arguments");
    int rc = require_supported(ctx, *n);
    if (rc) return rc;
    if (count == 0) return RN_OK;
    for (int32_t v = 0; v < count; ++v)
        for (int32_t j = 0; j < n->P; ++j)
            if (!in_domain(*n, j, x[(size_t)v * n->P + j]))
                return fail(ctx, RN_EINVAL, "vector %d: parameter %d is outside its domain", v, j);
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    const size_t xs = (size_t)count * n->P;
    const size_t ts = (size_t)count * n->C * n->T * n->N;
    RN_CUDA(ctx, ctx->xbuf.reserve(xs));
    RN_CUDA(ctx, ctx->sbuf.reserve((size_t)count));
    if (traj) RN_CUDA(ctx, ctx->tbuf.reserve(ts));
    RN_CUDA(ctx, cudaMemcpyAsync(ctx->xbuf.p, x, xs, cudaMemcpyHostToDevice, ctx->stream));
    if ((rc = evaluate_device_impl(ctx, *n, count, ctx->xbuf.p, n->P, ctx->sbuf.p, nullptr,
                                   traj ? ctx->tbuf.p : nullptr)))
        return rc;
    RN_CUDA(ctx, cudaMemcpyAsync(score, ctx->sbuf.p, sizeof(int32_t) * (size_t)count,
                                 cudaMemcpyDeviceToHost, ctx->stream));
    if (traj)
        RN_CUDA(ctx, cudaMemcpyAsync(traj, ctx->tbuf.p, ts, cudaMemcpyDeviceToHost, ctx->stream));
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return RN_OK;
}

int rn_evaluate_device(rn_ctx *ctx, int32_t net, int32_t count, const int8_t *x_dev,
                       int32_t *score_dev, uint8_t *traj_dev)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    Network *n = get_net(ctx, net);
    if (!n) return fail(ctx, RN_EINVAL, "unknown network %d", net);
    if (!n->has_tc) return fail(ctx, RN_ESTATE, "network %d has no time course", net);
    if (count < 0 || (count > 0 && (!x_dev || !score_dev)))
        return fail(ctx, RN_EINVAL, "bad arguments");
    int rc = require_supported(ctx, *n);
    if (rc) return rc;
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    if (count > 0) {
        char why[256];
        const size_t c = (size_t)count;
        if ((rc = check_device_span(x_dev, c * (size_t)n->P, ctx->device, "x_dev", why,
                                    sizeof why)) ||
            (rc = check_device_span(score_dev, c * sizeof(int32_t), ctx->device, "score_dev",
                                    why, sizeof why)) ||
            (traj_dev && (rc = check_device_span(traj_dev, c * (size_t)n->C * (size_t)n->T *
                                                               (size_t)n->N,
                                                 ctx->device, "traj_dev", why, sizeof why))))
            return fail(ctx, rc, "%s", why);
    }
    return evaluate_device_impl(ctx, *n, count, x_dev, n->P, score_dev, nullptr, traj_dev);
}

int rn_get_chain_state(rn_ctx *ctx, int32_t net, int8_t *x_cur, int32_t *d_cur, int8_t *x_best,
                       int32_t *d_best, int64_t *counters, int64_t *step)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    Network *n = get_net(ctx, net);
    if (!n) return fail(ctx, RN_EINVAL, "unknown network %d", net);
    if (!n->chains_valid) return fail(ctx, RN_ESTATE, "network %d has no chains", net);
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    const DevChains ch = n->chains();
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    int rc = check_device_flag(ctx);
    if (rc) return rc;
    if (x_cur && (rc = download_rows(ctx, *n, x_cur, ch.x_cur))) return rc;
    if (x_best && (rc = download_rows(ctx, *n, x_best, ch.x_best))) return rc;
    if (d_cur)
        RN_CUDA(ctx, cudaMemcpyAsync(d_cur, ch.d_cur, sizeof(int32_t) * (size_t)ch.n,
                                     cudaMemcpyDeviceToHost, ctx->stream));
    if (d_best)
        RN_CUDA(ctx, cudaMemcpyAsync(d_best, ch.d_best, sizeof(int32_t) * (size_t)ch.n,
                                     cudaMemcpyDeviceToHost, ctx->stream));
    if (counters)
        RN_CUDA(ctx, cudaMemcpyAsync(counters, ch.cnt, sizeof(int64_t) * 3 * (size_t)ch.n,
                                     cudaMemcpyDeviceToHost, ctx->stream));
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (step) *step = n->step;
    return RN_OK;
}

int rn_get_stats(rn_ctx *ctx, int32_t net, int64_t stats[5])
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    if (!stats) return fail(ctx, RN_EINVAL, "stats is NULL");
    Network *n = get_net(ctx, net);
    if (!n) return fail(ctx, RN_EINVAL, "unknown network %d", net);
    if (!n->chains_valid) return fail(ctx, RN_ESTATE, "network %d has no chains", net);
    const int32_t n_chains = n->chains().n;
    std::vector<int64_t> cnt((size_t)3 * (size_t)n_chains);
    int64_t step = 0;
    const int rc = rn_get_chain_state(ctx, net, nullptr, nullptr, nullptr, nullptr, cnt.data(), &step);
    if (rc) return rc;
    int64_t sum[3] = {0, 0, 0};
    for (size_t c = 0; c < (size_t)n_chains; ++c)
        for (int k = 0; k < 3; ++k) sum[k] += cnt[3 * c + (size_t)k];
    for (int k = 0; k < 3; ++k) stats[k] = sum[k];
    stats[3] = n_chains;
    stats[4] = step;
    return RN_OK;
}

int rn_set_chain_state(rn_ctx *ctx, int32_t net, int32_t n_chains, uint64_t seed,
                       const int8_t *x_cur, const int32_t *d_cur, const int8_t *x_best,
                       const int32_t *d_best, const int64_t *counters, int64_t step)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    Network *n = get_net(ctx, net);
    if (!n) return fail(ctx, RN_EINVAL, "unknown network %d", net);
    if (!n->has_tc) return fail(ctx, RN_ESTATE, "network %d has no time course", net);
    if (n_chains < 1 || !x_cur || !d_cur || !x_best || !d_best || !counters || step < 0)
        return fail(ctx, RN_EINVAL, "bad arguments");
    int rc = require_supported(ctx, *n);
    if (rc) return rc;
    for (int32_t c = 0; c < n_chains; ++c) {
        if ((rc = check_vector(ctx, *n, x_cur + (size_t)c * n->P, c))) return rc;
        if ((rc = check_vector(ctx, *n, x_best + (size_t)c * n->P, c))) return rc;
    }
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    n->chains_valid = false;
    if ((rc = alloc_chains(ctx, *n, n_chains))) return rc;
    const DevChains ch = n->chains();
    if ((rc = upload_rows(ctx, *n, ch.x_cur, x_cur, n_chains))) return rc;
    if ((rc = upload_rows(ctx, *n, ch.x_best, x_best, n_chains))) return rc;
    RN_CUDA(ctx, cudaMemcpyAsync(ch.d_cur, d_cur, sizeof(int32_t) * (size_t)n_chains,
                                 cudaMemcpyHostToDevice, ctx->stream));
    RN_CUDA(ctx, cudaMemcpyAsync(ch.d_best, d_best, sizeof(int32_t) * (size_t)n_chains,
                                 cudaMemcpyHostToDevice, ctx->stream));
    RN_CUDA(ctx, cudaMemcpyAsync(ch.cnt, counters, sizeof(int64_t) * 3 * (size_t)n_chains,
                                 cudaMemcpyHostToDevice, ctx->stream));
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    n->seed = seed;
    n->step = step;
    n->chains_valid = true;
    ctx->gen++;
    return RN_OK;
}

int rn_synchronize(rn_ctx *ctx)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return check_device_flag(ctx);
}

}  // extern "C"
