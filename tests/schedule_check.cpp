// Host-side check of a launch group's run schedule (spg::schedule_runs):
// seeded groups of members with log-uniform tile counts (empty members too)
// over grids of 1..2432 blocks.  Exits non-zero on the first violated
// property and prints one line per case: members, blocks, piece, tiles, runs,
// largest block work over the average (work = tiles + one set-up per run).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <random>
#include <vector>

#include "spegg_engine.h"

static int fail(int c, const char *what) {
    std::printf("FAIL case %d: %s\n", c, what);
    return 1;
}

int main() {
    std::mt19937 rng(20160329u);
    for (int c = 0; c < 300; ++c) {
        const uint32_t M = 1 + rng() % 400;
        const uint32_t G = c % 3 == 0 ? 152u * (1u + rng() % 16u) : 1u + rng() % 800u;
        const uint32_t piece = 1 + rng() % 64;
        std::vector<uint32_t> tiles(M);
        for (uint32_t &t : tiles) {
            const double u = (double)(rng() % 1000000u) / 1e6;
            t = rng() % 11u == 0 ? 0u : (uint32_t)std::exp(u * std::log(2000.0));
        }
        std::vector<spg::Run> runs;
        std::vector<uint32_t> br;
        spg::schedule_runs(tiles, G, piece, runs, br);
        if (br.size() != (size_t)G + 1 || br[0] != 0 || br[G] != runs.size()) return fail(c, "block offsets");
        std::vector<uint64_t> tstart(M + 1, 0);
        for (uint32_t m = 0; m < M; ++m) tstart[m + 1] = tstart[m] + tiles[m];
        const uint64_t T = tstart[M];
        std::vector<std::vector<uint8_t>> cov(M);
        for (uint32_t m = 0; m < M; ++m) cov[m].assign(tiles[m], 0);
        std::vector<uint32_t> nruns(M, 0);
        std::vector<std::vector<std::pair<uint32_t, uint32_t>>> shares(M);  // (tile0, share)
        double work_max = 0, work_sum = 0;
        uint64_t units = 0;
        for (uint32_t m = 0; m < M; ++m) units += tiles[m] ? tiles[m] + 1u : 0u;
        for (uint32_t b = 0; b < G; ++b) {
            if (br[b] > br[b + 1]) return fail(c, "block offsets decrease");
            double w = 0;
            uint64_t last = 0;
            for (uint32_t i = br[b]; i < br[b + 1]; ++i) {
                const spg::Run &r = runs[i];
                if (r.seg >= M || r.count == 0 || (uint64_t)r.tile0 + r.count > tiles[r.seg]) return fail(c, "run bounds");
                const uint64_t at = tstart[r.seg] + r.tile0;
                if (i > br[b] && at < last) return fail(c, "a block's runs go back in the member list");
                last = at + r.count;
                for (uint32_t t = r.tile0; t < r.tile0 + r.count; ++t)
                    if (cov[r.seg][t]++) return fail(c, "tile formed twice");
                ++nruns[r.seg];
                shares[r.seg].push_back({r.tile0, r.share});
                w += r.count + 1.0;
            }
            work_max = std::max(work_max, w);
            work_sum += w;
        }
        for (uint32_t m = 0; m < M; ++m)
            for (uint8_t v : cov[m])
                if (v != 1) return fail(c, "tile not formed");
        for (const spg::Run &r : runs)
            if (r.shares != nruns[r.seg]) return fail(c, "shares is not the member's run count");
        for (uint32_t m = 0; m < M; ++m) {
            std::sort(shares[m].begin(), shares[m].end());
            for (size_t i = 0; i < shares[m].size(); ++i)
                if (shares[m][i].second != i) return fail(c, "shares not numbered in tile order");
        }
        // rounds of G pieces of equal units (+-1), each piece at most one
        // uncounted set-up (a member continued from the previous piece)
        const uint64_t rounds = std::max<uint64_t>(1, T / ((uint64_t)G * piece));
        if (work_max > (double)units / G + 3.0 * rounds + 1.0) return fail(c, "block work above the bound");
        // the launch table holds one run per member plus one per piece: G
        // pieces, or pieces of min_piece tiles or more
        if (runs.size() > (size_t)M + std::max<uint64_t>(G, T / piece)) return fail(c, "more runs than the table holds");
        std::printf("%u %u %u %llu %zu %.4f\n", M, G, piece, (unsigned long long)T, runs.size(),
                    work_sum > 0 ? work_max / (work_sum / G) : 1.0);
    }
    std::printf("ok\n");
    return 0;
}
