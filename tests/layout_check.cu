// Host-side check of a network's table layout (no GPU is used): reads a
// network (int32 N, int32 E, int32 src[E], int32 dst[E]) from argv[1], runs the
// library's layout builder and prints
//   supported lanes npl two_copies rows wavefronts lower_bound_one_copy
// on one line, or a message and exit status 1 when an invariant fails:
//  - every edge sits in exactly one table entry, in the lane and slot of its
//    destination node, and edge_pos names that entry;
//  - every entry's code address (either copy, or a padding read) lies inside
//    the code region of the block's shared memory.
// wavefronts counts the code gather of one update step on the block path: per
// slot, warp and row, the largest number of distinct 4-byte words one bank
// serves.  lower_bound_one_copy is what any placement of the rows over a single
// copy of the codes needs: per slot and warp, the most distinct words one bank
// holds, and at least one wavefront per row.
#include <cstdio>
#include <map>
#include <set>
#include <vector>

#include "../paper_2506_19866_gb300/csrc/rn_context.h"

namespace rn {
void build_layout(Network &n);
}

static int fail(const char *what, long a)
{
    std::printf("invariant failed: %s (%ld)\n", what, a);
    return 1;
}

int main(int argc, char **argv)
{
    if (argc < 2) return 2;
    FILE *f = std::fopen(argv[1], "rb");
    if (!f) return 2;
    int32_t N = 0, E = 0;
    if (std::fread(&N, 4, 1, f) != 1 || std::fread(&E, 4, 1, f) != 1) return 2;
    rn::Network n;
    n.N = N;
    n.E = E;
    n.P = 3 * E + 3 * N;
    n.src.resize((size_t)E);
    n.dst.resize((size_t)E);
    n.fast.assign((size_t)N, 0);
    if (std::fread(n.src.data(), 4, (size_t)E, f) != (size_t)E ||
        std::fread(n.dst.data(), 4, (size_t)E, f) != (size_t)E)
        return 2;
    std::fclose(f);
    rn::build_layout(n);
    if (!n.supported || n.lanes != rn::kBlockLanes) {
        std::printf("supported %d lanes %d npl %d\n", (int)n.supported, n.lanes, n.npl);
        return 0;
    }
    const int L = n.lanes, W = L / 32, npl = n.npl;
    const bool two = rn::block_path_two_copies(n.D, npl, N);
    const uint32_t code_bytes = rn::block_code_bytes(npl) * (two ? 2u : 1u);
    std::vector<int> seen((size_t)E, 0);
    long rows = 0, wavefronts = 0, lower = 0;
    for (int k = 0; k < npl; ++k)
        for (int wg = 0; wg < W; ++wg) {
            const int d4 = n.warp_d4[(size_t)k * W + wg];
            std::map<int, std::set<int>> one_copy;   // bank -> first-copy words of the group's edges
            for (int d = 0; d < d4; ++d) {
                std::map<int, std::set<int>> banks;
                for (int l = 0; l < 32; ++l) {
                    const int t = 32 * wg + l;
                    const int v = d < n.dtab ? n.edge_id[((size_t)k * n.dtab + d) * L + t] : -1;
                    long byte;
                    if (v >= 0) {
                        const int e = v & ~rn::kCodeCopy2;
                        if (e >= E) return fail("edge index", e);
                        seen[(size_t)e]++;
                        if (n.dst[(size_t)e] != n.q_node[(size_t)t * npl + k])
                            return fail("edge outside its node's lane and slot", e);
                        const int pos = n.edge_pos[(size_t)e];
                        if ((pos >> 16) != t || ((pos >> 8) & 0xff) != k || (pos & 0xff) != d)
                            return fail("edge_pos", e);
                        const uint32_t q = (uint32_t)n.node_q[(size_t)n.src[(size_t)e]];
                        byte = (v & rn::kCodeCopy2)
                                   ? (long)(rn::block_code_bytes(npl) + 4u * rn::code_word2(q >> 1) +
                                            2u * (q & 1u))
                                   : 2L * q;
                        if ((v & rn::kCodeCopy2) && !two) return fail("second copy without one", e);
                        one_copy[(int)(q >> 1) & 31].insert((int)(q >> 1));
                    } else {
                        byte = -1L - v;
                    }
                    if (byte < 0 || byte + 2 > (long)code_bytes) return fail("code address", byte);
                    banks[(int)(byte >> 2) & 31].insert((int)(byte >> 2));
                }
                size_t m = 1;
                for (auto &b : banks) m = b.second.size() > m ? b.second.size() : m;
                wavefronts += (long)m;
                ++rows;
            }
            size_t mb = 0;
            for (auto &b : one_copy) mb = b.second.size() > mb ? b.second.size() : mb;
            lower += (long)(mb > (size_t)d4 ? mb : (size_t)d4);
        }
    for (int e = 0; e < E; ++e)
        if (seen[(size_t)e] != 1) return fail("edge placed other than once", e);
    std::printf("supported 1 lanes %d npl %d two_copies %d rows %ld wavefronts %ld "
                "lower_bound_one_copy %ld\n",
                L, npl, (int)two, rows, wavefronts, lower);
    return 0;
}
