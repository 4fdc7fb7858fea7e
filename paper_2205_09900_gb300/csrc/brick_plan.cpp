// brick_plan.cpp -- light-cone tile schedule of the brickwork dual sweep.
//
// A side is a sequence of layers; layer t applies gates j = 0..m-1 on bits
// (tau, tau+1 mod N), tau = 2j + p_t, where p_t alternates.  A tile holds K
// bits forming a contiguous cyclic arc of the ring that contains the `low`
// lowest physical bits (so that loading a tile reads runs of 2^low contiguous
// amplitudes).  Greedy schedule: each pass takes the arc that can apply the
// most not-yet-applied gates whose bits lie in the arc and whose
// predecessors (gates of the previous layer sharing a bit) are applied.
#include <algorithm>
#include <cstring>

#include "brick.h"

namespace fpk {

BrickHostPlan make_brick_plan(int n, int l, int tile_bits, int low_bits) {
    BrickHostPlan P;
    BrickDev &d = P.dev;
    std::memset(&d, 0, sizeof d);
    d.n = n;
    d.l = l;
    d.m = l - 1;
    d.N = 2 * d.m;
    d.cut = n / 2;
    d.n_layers[0] = d.cut;
    d.n_layers[1] = n - 1 - d.cut;
    d.delta_par[0] = 0;        // qubit 0 is idle where bond 0 (parity 1 positions) is not
    d.delta_par[1] = n % 2;    // qubit n-1 is idle where bond n-2 is not
    const int N = d.N, m = d.m;
    d.tile_bits = tile_bits >= N ? 0 : tile_bits;
    if (d.tile_bits == 0) return P;
    const int K = tile_bits;
    // candidate arcs: those holding the low bits first (coalesced tile loads);
    // every arc when none of those can make progress
    std::vector<uint32_t> arcs, all_arcs;
    for (int s = 0; s < N; ++s) {
        uint32_t mask = 0;
        for (int i = 0; i < K; ++i) mask |= 1u << ((s + i) % N);
        uint32_t low = (1u << std::min(low_bits, K)) - 1u;
        if ((mask & low) == low) arcs.push_back(mask);
        all_arcs.push_back(mask);
    }
    for (int side = 0; side < 2; ++side) {
        const int L = d.n_layers[side];
        d.pass_off[side] = (int)P.passes.size();
        std::vector<char> done((size_t)L * m, 0);
        auto par = [&](int t) { return (brick_bond(d, side, t) + 1) % 2; };
        auto bits = [&](int t, int j) {
            int tau = 2 * j + par(t);
            return (1u << tau) | (1u << ((tau + 1) % N));
        };
        size_t left = (size_t)L * m;
        while (left > 0) {
            uint32_t best_mask = 0;
            std::vector<int> best;
            for (int round = 0; round < 2 && best.empty(); ++round)
            for (uint32_t S : (round == 0 ? arcs : all_arcs)) {
                std::vector<char> got((size_t)L * m, 0);
                std::vector<int> list;
                for (int t = 0; t < L; ++t)
                    for (int j = 0; j < m; ++j) {
                        size_t id = (size_t)t * m + j;
                        if (done[id]) continue;
                        uint32_t bj = bits(t, j);
                        if ((bj & S) != bj) continue;
                        bool ok = true;
                        if (t > 0)
                            for (int jj = 0; jj < m && ok; ++jj)
                                if ((bits(t - 1, jj) & bj) && !done[(size_t)(t - 1) * m + jj] &&
                                    !got[(size_t)(t - 1) * m + jj])
                                    ok = false;
                        if (ok) { got[id] = 1; list.push_back((int)id); }
                    }
                if (list.size() > best.size()) { best = list; best_mask = S; }
            }
            if (best.empty()) break;   // cannot happen for K >= 2
            BrickPass ps;
            ps.gate_off = (int)P.gates.size();
            ps.n_gates = (int)best.size();
            ps.smask = best_mask;
            int loc[32];
            for (int b = 0, k = 0; b < N; ++b) if (best_mask & (1u << b)) loc[b] = k++;
            for (int id : best) {
                int t = id / m, j = id % m, tau = 2 * j + par(t);
                BrickGate g;
                g.layer = (uint8_t)t;
                g.j = (uint8_t)j;
                g.a = (uint8_t)loc[tau];
                g.b = (uint8_t)loc[(tau + 1) % N];
                P.gates.push_back(g);
                done[id] = 1;
            }
            left -= best.size();
            P.passes.push_back(ps);
        }
        d.n_passes[side] = (int)P.passes.size() - d.pass_off[side];
    }
    return P;
}

}  // namespace fpk
