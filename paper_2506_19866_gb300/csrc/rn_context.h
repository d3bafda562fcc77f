// rn_context.h -- host-side state of a library context (networks, chains,
// schedule tables, batched-launch state) shared by the translation units
// that implement the C ABI.
#pragma once

#include <cstdarg>
#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "../../include/rnanneal.h"
#include "rn_launch.h"

namespace rn {

// Device buffer owned by the context.
template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    cudaError_t alloc(size_t count)
    {
        release();
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc(&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        n = count;
        return cudaSuccess;
    }
    cudaError_t reserve(size_t count)
    {
        return count <= n ? cudaSuccess : alloc(count);
    }
    cudaError_t upload(const std::vector<T> &v)
    {
        cudaError_t e = alloc(v.size());
        if (e != cudaSuccess) return e;
        if (v.empty()) return cudaSuccess;
        return cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    }
};

struct Network {
    int32_t N = 0, E = 0, P = 0;
    std::vector<int32_t> src, dst;
    std::vector<uint8_t> fast, frozen;
    std::vector<int8_t> frozen_val;
    bool has_frozen = false;
    bool sync = false;                // synchronous update scheme (rn_set_update_scheme)
    // lane / slot layout
    int npl = 0, dtab = 0;
    int lanes = 32;                     // threads per chain: 32, or kBlockLanes above 512 nodes
    int D[kMaxSlots] = {};
    std::vector<int32_t> node_q, edge_id, edge_pos, free_list, in_ptr, in_edges, out_ptr,
        out_edges;
    std::vector<int16_t> q_node;
    std::vector<uint8_t> edge_q2;
    std::vector<uint8_t> warp_d4;       // block path: [npl][lanes / 32] rows gathered per warp
    bool supported = false;
    // device copies
    DevBuf<int32_t> d_edge_id, d_edge_pos, d_node_q, d_src, d_dst, d_free, d_in_ptr, d_in_edges,
        d_out_ptr, d_out_edges;
    DevBuf<int16_t> d_q_node;
    DevBuf<uint8_t> d_edge_q2, d_fast, d_frozen, d_warp_d4;
    DevBuf<int8_t> d_frozen_val;
    // time course: conditions are simulated cg at a time, G groups
    bool has_tc = false;
    int32_t C = 0, T = 0, cg = 1, G = 0;
    int d0 = -1, d1 = -1;               // register capacities of the anneal kernel
    int64_t max_score = 0;
    int64_t n_obs = 0;                  // observed entries of the time course
    DevBuf<uint16_t> d_init_code, d_out_bits;
    DevBuf<uint32_t> d_obs, d_init_s4, d_movable;
    std::vector<uint32_t> movable_h;    // host copy of d_movable
    bool async_ = false;                // asynchronous update scheme (rn_set_update_scheme)
    DevBuf<uint32_t> d_movable_t;       // [G][T][lanes][npl]: the step's selected node
    DevBuf<int32_t> d_async_sel;        // [C][T] the selection itself
    // chains
    int32_t n_chains = 0;
    int32_t pstride = 0;
    uint64_t seed = 0;
    int64_t step = 0;
    bool chains_valid = false;
    DevBuf<int8_t> d_x_cur, d_x_best;
    DevBuf<int32_t> d_d_cur, d_d_best;
    DevBuf<int64_t> d_cnt;

    DevNet dev() const
    {
        DevNet n{};
        n.N = N; n.E = E; n.P = P; n.n_free = (int32_t)free_list.size();
        n.C = C; n.T = T; n.G = G;
        n.npl = npl; n.cg = cg; n.dtab = dtab; n.lanes = lanes;
        n.sync = (sync || async_) ? 1 : 0;
        n.async = async_ ? 1 : 0;
        n.movable_t = async_ ? d_movable_t.p : nullptr;
        n.async_sel = async_ ? d_async_sel.p : nullptr;
        for (int k = 0; k < kMaxSlots; ++k) n.D[k] = D[k];
        n.edge_id = d_edge_id.p; n.edge_q2 = d_edge_q2.p; n.edge_pos = d_edge_pos.p;
        n.warp_d4 = warp_d4.empty() ? nullptr : d_warp_d4.p;
        n.node_q = d_node_q.p; n.q_node = d_q_node.p; n.src = d_src.p; n.dst = d_dst.p;
        n.fast = d_fast.p; n.free_list = d_free.p;
        n.in_ptr = d_in_ptr.p; n.in_edges = d_in_edges.p;
        n.out_ptr = d_out_ptr.p; n.out_edges = d_out_edges.p;
        n.frozen = has_frozen ? d_frozen.p : nullptr;
        n.frozen_val = has_frozen ? d_frozen_val.p : nullptr;
        n.init_code = d_init_code.p; n.out_bits = d_out_bits.p; n.obs = d_obs.p;
        n.init_s4 = d_init_s4.p; n.movable = d_movable.p;
        return n;
    }
    DevChains chains() const
    {
        DevChains c{};
        c.n = n_chains; c.pstride = pstride; c.seed = seed;
        c.x_cur = d_x_cur.p; c.x_best = d_x_best.p;
        c.d_cur = d_d_cur.p; c.d_best = d_d_best.p; c.cnt = d_cnt.p;
        return c;
    }
};


struct SchedCache {
    bool valid = false;
    double T0 = 0, alpha = 0;
    int64_t iters = 0, l0 = 0, l1 = -1, cap = 0;
    DevBuf<uint32_t> thr;
    DevBuf<int32_t> off, len;
};

// Device descriptors of a batched launch over every network with chains, the
// autotuned configuration, and the CUDA graph that replays the launch.
constexpr int kBatchCandidates = 10;
struct BatchState {
    bool valid = false;
    uint64_t gen = 0;                 // context generation it was built for
    std::vector<int> order;           // context network ids, most work per chain first
    int32_t total = 0;
    int32_t total_big = 0;            // chains of networks on the shared-memory tables
    int32_t large = 0;                // large-region warps per block
    bool all_large = false;           // every warp gets a large region (a tuning candidate)
    uint32_t region_small = 0;        // region of a small (register-table) warp
    DevBuf<rn::DevNet> nets;
    DevBuf<rn::DevChains> chains;
    DevBuf<int64_t> g0;
    DevBuf<int32_t> item_net, item_chain, path;
    std::vector<int32_t> host_path;   // chosen table path per network (batch order)
    uint32_t region_bytes = 0;
    int wpb = 4, grid = 0;
    bool tuned = false;
    bool g0_synced = false;           // device g0 equals the host step counters
    bool phased = false;              // one launch per table path (candidates 8, 9)
    std::vector<BatchPhase> phases;   // of a phased launch, in launch order
    std::vector<int32_t> phase_wpb;   // warps per block of each phase (by table path)
    double tune_ms[kBatchCandidates] = {};   // trial times of the candidates
    int32_t force = -1;               // candidate pinned by rn_batch_tune (-1: autotune)
    int32_t cfg = 0;                  // candidate in use
    // graph of [queue reset, batched kernel, step advance]
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t graph_sweeps = -1;
    int32_t graph_early = 0;          // early_reject flag the graph was captured with
    void drop_graph()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        graph_sweeps = -1;
    }
    ~BatchState() { drop_graph(); }
};

}  // namespace rn

namespace rn {

// Learned proposal screen of one network: an MLP on the one-hot parameter
// vector, y = b3 + w3 . relu(b2 + W2^T relu(b1 + W1^T onehot(x))).
struct Mlp {
    int32_t net = -1;
    int32_t P = 0, pstride = 0;
    int32_t H1 = 0, H2 = 0;
    int32_t D = 0, Dp = 0;              // one-hot width, padded to a multiple of 128
    double scale = 1.0;                 // logged target = score * scale (1 / observed entries)
    DevBuf<int32_t> row_base;           // [P] one-hot row of value v of parameter j: row_base[j] + v
    // FP32 masters, gradients and Adam moments, each laid out
    // [W1 (Dp x H1) | b1 (H1) | W2 (H1 x H2) | b2 (H2) | w3 (H2) | b3]
    size_t n_theta = 0;
    DevBuf<float> theta, grad, adam_m, adam_v;
    int64_t adam_t = 0;
    DevBuf<float> adam_c;               // [2 x steps] Adam bias corrections of one training call
    DevBuf<uint32_t> train_k;           // the step within a training call (advanced on the device)
    // BF16 copies (bit patterns): W1T [H1][Dp], W1b [Dp][H1], W2T [H2][H1], W2b [H1][H2]
    DevBuf<uint16_t> W1T, W1b, W2T, W2b;
    // training set (ring of logged pairs)
    int64_t cap = 0, count = 0, head = 0;
    DevBuf<int8_t> set_x;               // [cap][pstride]
    DevBuf<float> set_y;                // [cap]
    // batch scratch for up to Bcap rows
    int32_t Bcap = 0;
    DevBuf<uint16_t> oh, ohT, h1, h1T, h2, dh2, dh2T, dh1, dh1T;
    DevBuf<float> part, y, dy, tgt, colpart;
    DevBuf<int32_t> idx;
    DevBuf<int8_t> xrows;               // [Bcap][pstride] host rows staged on the device
    DevBuf<double> loss;
    // screened annealing: layer-1 pre-activation of every chain's x_cur and
    // the per-step candidate buffers
    int32_t chains = 0, K = 0, top = 0;
    bool a1_valid = false;              // A1 holds the pre-activations of x_cur at
    uint64_t a1_gen = 0;                // context generation a1_gen and step a1_step
    int64_t a1_step = -1;
    DevBuf<float> A1;                   // [chains][H1]
    DevBuf<uint16_t> hc;                // [Mc][H1] candidate hidden rows (bf16), hidden-row mode 1
    DevBuf<int2> rows;                  // [Mc] W1 rows (new, old) per candidate, hidden-row mode 0
    int32_t hidden_mode = 1;            // 0: hidden rows formed in the GEMM; 1: through memory
    DevBuf<float> pc;                   // [Mc][H2 / 64] candidate layer-2 partials
    DevBuf<int32_t> cand;               // [chains][K] (j << 8) | (v & 255), -1 = null
    DevBuf<uint16_t> emb_oh;            // [kEmbedRows][Dp] one-hot rows of chains (large P)
    DevBuf<float> emb_out;              // [kEmbedRows][H1] their layer-1 products

    size_t off_b1() const { return (size_t)Dp * H1; }
    size_t off_W2() const { return off_b1() + H1; }
    size_t off_b2() const { return off_W2() + (size_t)H1 * H2; }
    size_t off_w3() const { return off_b2() + H2; }
    size_t off_b3() const { return off_w3() + H2; }
};

// Launches of the networks outside the batched launch.  Each network gets a
// work-item counter and a region of per-chain chunk counters of its own, so its
// launch may run beside the others: on side streams that fork from the
// context's stream and join back into it within one rn_anneal call, so that
// the launches of one network fill the tails of the others' persistent grids.
constexpr int kSideStreams = 4;
struct SideLaunch {
    DevBuf<unsigned int> queue;   // one counter per separate network
    DevBuf<int32_t> done;         // one region of n_chains counters per network
    cudaStream_t streams[kSideStreams] = {};
    cudaEvent_t join[kSideStreams] = {};
    cudaEvent_t fork = nullptr;
    bool ready = false;
    SideLaunch() = default;
    SideLaunch(const SideLaunch &) = delete;
    SideLaunch &operator=(const SideLaunch &) = delete;
    cudaError_t create()
    {
        if (ready) return cudaSuccess;
        cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        for (int k = 0; e == cudaSuccess && k < kSideStreams; ++k) {
            e = cudaStreamCreateWithFlags(&streams[k], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            destroy();
            return e;
        }
        ready = true;
        return cudaSuccess;
    }
    void destroy()
    {
        for (int k = 0; k < kSideStreams; ++k) {
            if (streams[k]) {
                cudaStreamSynchronize(streams[k]);
                cudaStreamDestroy(streams[k]);
            }
            if (join[k]) cudaEventDestroy(join[k]);
            streams[k] = nullptr;
            join[k] = nullptr;
        }
        if (fork) cudaEventDestroy(fork);
        fork = nullptr;
        ready = false;
    }
    ~SideLaunch() { destroy(); }
};

}  // namespace rn

struct rn_ctx {
    int device = 0;
    int64_t launches = 0;
    uint64_t gen = 1;                 // bumped whenever networks or chains change
    rn::BatchState batch;
    rn::SchedCache cache;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    std::vector<std::unique_ptr<rn::Network>> nets;
    std::vector<std::unique_ptr<rn::Mlp>> mlps;
    rn::DevBuf<uint32_t> thr;
    rn::DevBuf<int32_t> thr_off, thr_len;
    rn::DevBuf<int32_t> status;
    rn::DevBuf<int32_t> winner;
    rn::DevBuf<unsigned int> queue;   // work-item counters of the batched launch
    rn::DevBuf<int32_t> done;         // chunks finished per chain in the batched launch
    rn::SideLaunch side;              // the networks launched on their own
    rn::DevBuf<int32_t> dev_err;      // set by a kernel whose wait gave up
    rn::DevBuf<int8_t> xbuf;
    rn::DevBuf<int32_t> sbuf;
    rn::DevBuf<uint8_t> tbuf;
};

namespace rn {

// Helpers of rn_api.cu used by the other ABI translation units.
int fail(rn_ctx *ctx, int code, const char *fmt, ...);
int cuda_fail(rn_ctx *ctx, cudaError_t e, const char *what);
Network *get_net(rn_ctx *ctx, int32_t id);
int domain_of(const Network &n, int32_t j, int8_t vals[6]);
int check_vector(rn_ctx *ctx, const Network &n, const int8_t *x, int64_t which);
int check_device_flag(rn_ctx *ctx);
int require_supported(rn_ctx *ctx, const Network &n);
int evaluate_device_impl(rn_ctx *ctx, Network &n, int32_t count, const int8_t *x, int64_t xstride,
                         int32_t *score, int32_t *score2, uint8_t *traj);
int thresholds_for(rn_ctx *ctx, const rn_schedule &s, int64_t l0, int64_t l1, int64_t cap,
                   DevSched &sc, bool &cached);

}  // namespace rn

#define RN_CUDA(ctx, call)                                         \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return rn::cuda_fail((ctx), e_, #call); \
    } while (0)
