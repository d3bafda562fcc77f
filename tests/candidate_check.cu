// Host check of pick_alternative (rn_device.cuh), GetCandidate's choice of a new
// value: for every parameter kind, fast flag, current value and constraint case
// that can arise, and for many acceptance-independent draws r1, it must return
// the value that a walk over the domain's listed values picks (the domains of
// Sections 2.1-2.2, the constraints of Section 2.5.3).  Prints the number of
// cases and exits 1 on the first mismatch.
#include <cstdint>
#include <cstdio>

#include "../paper_2506_19866_gb300/csrc/rn_device.cuh"

static int listed_domain(int kind, bool fast, int (&vals)[6])
{
    static const int w[] = {0, 1, 2}, p[] = {-1, 0, 1}, t[] = {1, 2}, uf[] = {10, 11, 12},
                     us[] = {1, 2, 3, 4, 5, 6}, m[] = {0, 1, 2}, d[] = {1, 2};
    const int *src;
    int n;
    switch (kind) {
    case 0: src = w; n = 3; break;
    case 1: src = p; n = 3; break;
    case 2: src = t; n = 2; break;
    case 3: src = fast ? uf : us; n = fast ? 3 : 6; break;
    case 4: src = m; n = 3; break;
    default: src = d; n = 2; break;
    }
    for (int k = 0; k < n; ++k) vals[k] = src[k];
    return n;
}

static bool walk(int kind, bool fast, int cur, bool b0, bool ball, uint32_t r1, int &v)
{
    int vals[6], alts[6], n_alt = 0;
    const int n = listed_domain(kind, fast, vals);
    if (!ball)
        for (int k = 0; k < n; ++k)
            if (vals[k] != cur && !(b0 && vals[k] == 0)) alts[n_alt++] = vals[k];
    if (n_alt == 0) return false;
    v = alts[(uint32_t)(((uint64_t)r1 * (uint32_t)n_alt) >> 32)];
    return true;
}

int main()
{
    uint64_t state = 0x9E3779B97F4A7C15ull;   // splitmix64 stream of draws
    long cases = 0;
    for (int kind = 0; kind < 6; ++kind)
        for (int fast = 0; fast < 2; ++fast) {
            int vals[6];
            const int n = listed_domain(kind, fast, vals);
            for (int ci = 0; ci < n; ++ci)
                for (int b0 = 0; b0 < 2; ++b0)
                    for (int ball = 0; ball < 2; ++ball) {
                        const int cur = vals[ci];
                        // blocked0: a nonzero w whose edge is needed; blocked_all:
                        // a needed positive sign (the only cases GetCandidate forms)
                        if (b0 && !(kind == 0 && cur != 0)) continue;
                        if (ball && !(kind == 1 && cur == 1)) continue;
                        for (int k = 0; k < 100000; ++k) {
                            uint32_t r1;
                            if (k == 0) r1 = 0u;
                            else if (k == 1) r1 = 0xffffffffu;
                            else {
                                uint64_t z = (state += 0x9E3779B97F4A7C15ull);
                                z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
                                z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
                                r1 = (uint32_t)(z ^ (z >> 31));
                            }
                            int v1 = -99, v2 = -99;
                            const bool o1 = walk(kind, fast, cur, b0, ball, r1, v1);
                            const bool o2 = rn::pick_alternative(kind, fast, cur, b0, ball, r1, v2);
                            ++cases;
                            if (o1 != o2 || (o1 && v1 != v2)) {
                                std::printf("mismatch: kind %d fast %d cur %d blocked0 %d "
                                            "blocked_all %d r1 %u: %d %d / %d %d\n",
                                            kind, fast, cur, b0, ball, r1, (int)o1, v1, (int)o2,
                                            v2);
                                return 1;
                            }
                        }
                    }
        }
    std::printf("cases %ld\n", cases);
    return 0;
}
