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
#include <array>
#include <cstring>

#include "brick.h"

namespace fpk {

// Register windows inside one tile pass: windows are r consecutive ring
// positions of the tile's arc; greedy, each step takes the window that can
// apply the most remaining gates (in layer order, predecessors first).
static void schedule_registers(BrickHostPlan &P, BrickPass &ps, const int *ring, int K, int r, bool cyclic) {
    const int G = ps.n_gates;
    std::vector<int> rpos(32, -1);   // tile-local bit -> arc position
    for (int k = 0; k < K; ++k) rpos[ring[k]] = k;
    std::vector<char> done(G, 0);
    ps.rp_off = (int)P.rpasses.size();
    ps.rg_off = (int)P.rgates.size();
    int left = G;
    while (left > 0) {
        int best_c = -1;
        std::vector<std::pair<int, int>> best;   // (gate index, type)
        const int nwin = cyclic ? K : K - r + 1;
        for (int c = 0; c < nwin; ++c) {
            std::vector<char> got(G, 0);
            std::vector<std::pair<int, int>> list;
            for (int g = 0; g < G; ++g) {
                if (done[g]) continue;
                const BrickGate &bg = P.gates[ps.gate_off + g];
                int pa = rpos[bg.a], pb = rpos[bg.b];
                int i = cyclic ? (pa - c + K) % K : pa - c;
                if (cyclic ? pb != (pa + 1) % K : pb != pa + 1) continue;
                if (i < 0 || i > r - 2) continue;
                bool ok = true;
                for (int h = 0; h < g && ok; ++h) {       // earlier gates of the pass sharing a bit
                    const BrickGate &bh = P.gates[ps.gate_off + h];
                    if (bh.layer >= bg.layer) continue;
                    bool share = bh.a == bg.a || bh.a == bg.b || bh.b == bg.a || bh.b == bg.b;
                    if (share && !done[h] && !got[h]) ok = false;
                }
                if (ok) { got[g] = 1; list.push_back({g, i}); }
            }
            if (list.size() > best.size()) { best = list; best_c = c; }
        }
        if (best.empty()) break;
        RegPass rp;
        std::memset(&rp, 0, sizeof rp);
        rp.r = (uint8_t)r;
        for (int i = 0; i < r; ++i) rp.win[i] = (uint8_t)ring[(best_c + i) % K];
        for (int i = 0; i < r; ++i) rp.srt[i] = rp.win[i];
        std::sort(rp.srt, rp.srt + r);
        rp.n_gates = (uint8_t)best.size();
        rp.gate_off = (int16_t)P.rgates.size();
        for (auto &x : best) {
            RegGate rg;
            rg.type = (uint8_t)x.second;
            rg.slot = (uint8_t)x.first;
            P.rgates.push_back(rg);
            done[x.first] = 1;
        }
        left -= (int)best.size();
        P.rpasses.push_back(rp);
    }
    ps.n_rp = (int)P.rpasses.size() - ps.rp_off;
}

// Rank over GF(2) of up to 4 vectors of 4 bits.
static int rank4(uint32_t *v, int nv) {
    int r = 0;
    for (int bit = 3; bit >= 0 && r < nv; --bit) {
        int p = -1;
        for (int i = r; i < nv; ++i)
            if ((v[i] >> bit) & 1u) { p = i; break; }
        if (p < 0) continue;
        std::swap(v[r], v[p]);
        for (int i = 0; i < nv; ++i)
            if (i != r && ((v[i] >> bit) & 1u)) v[i] ^= v[r];
        ++r;
    }
    return r;
}

// The tile layout of one pass (BrickPass::swz): the lanes of a half-warp are
// consecutive groups t, whose bits 0-3 land on the 4 lowest tile bits outside
// the window; their 8-byte bank pairs (element index mod 16 after the
// swizzle) are distinct when those 4 bits' bank contributions are linearly
// independent.  Start from the fixed pattern (bit b -> b mod 4) and search
// (deterministic pseudo-random changes) until every window qualifies.
static void choose_swizzle(const BrickHostPlan &P, BrickPass &ps, int K) {
    for (int j = 0; j < 12; ++j) ps.swz[j] = (uint8_t)(1u << ((4 + j) % 4));
    if (K <= 4) return;
    auto bad = [&](const uint8_t *sw) {
        int cnt = 0;
        for (int w = 0; w < ps.n_rp; ++w) {
            const RegPass &rp = P.rpasses[ps.rp_off + w];
            uint32_t v[4];
            int nv = 0;
            for (int b = 0; b < K && nv < 4; ++b) {
                bool in = false;
                for (int k = 0; k < rp.r; ++k) in = in || rp.win[k] == b;
                if (!in) v[nv++] = b < 4 ? (1u << b) : sw[b - 4];
            }
            cnt += 4 - rank4(v, nv);
        }
        return cnt;
    };
    int best = bad(ps.swz);
    uint32_t x = 0x9E3779B9u ^ (uint32_t)ps.gate_off;
    for (int it = 0; it < 4000 && best > 0; ++it) {
        uint8_t trial[12];
        std::memcpy(trial, ps.swz, 12);
        x ^= x << 13; x ^= x >> 17; x ^= x << 5;
        trial[(x >> 4) % (uint32_t)(K - 4)] = (uint8_t)(x & 15u);
        const int v = bad(trial);
        if (v <= best) { best = v; std::memcpy(ps.swz, trial, 12); }
    }
}

BrickHostPlan make_brick_plan(int n, int l, int tile_bits, int low_bits, int win_bits, int kind) {
    BrickHostPlan P;
    BrickDev &d = P.dev;
    std::memset(&d, 0, sizeof d);
    d.n = n;
    d.l = l;
    d.m = l - 1;
    d.N = 2 * d.m;
    d.cut = n / 2;
    d.kind = kind;
    d.n_layers[0] = kind == 0 ? d.cut : 2 * d.cut;
    d.n_layers[1] = kind == 0 ? n - 1 - d.cut : 2 * (n - 1 - d.cut) + 2;
    d.delta_par[0] = 0;        // qubit 0 is idle where bond 0 (parity 1 positions) is not
    d.delta_par[1] = n % 2;    // qubit n-1 is idle where bond n-2 is not
    const int N = d.N, m = d.m;
    // tile_bits == N: the whole ring is one tile (one pass per side)
    d.tile_bits = tile_bits > N ? 0 : tile_bits;
    if (d.tile_bits == 0) return P;
    const int K = tile_bits;
    const bool whole = K == N;
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
        auto par = [&](int t) { return layer_parity(d, side, t); };
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
            std::memset(&ps, 0, sizeof ps);
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
            // ring order of the arc: start where the previous ring bit is outside it
            int ring[32], start = 0;
            for (int b = 0; b < N; ++b)
                if ((best_mask & (1u << b)) && !(best_mask & (1u << ((b + N - 1) % N)))) start = b;
            for (int k = 0; k < K; ++k) ring[k] = loc[(start + k) % N];
            if (whole) for (int k = 0; k < K; ++k) ring[k] = loc[k];
            schedule_registers(P, ps, ring, K, std::min(win_bits, K), whole);
            choose_swizzle(P, ps, K);
            P.passes.push_back(ps);
        }
        d.n_passes[side] = (int)P.passes.size() - d.pass_off[side];
    }
    return P;
}

// Bank-pair index (8-byte banks of a 128-byte line) of an operand byte address.
static int bank8(uint32_t a) { return (int)((a >> 3) & 15u); }

// The store order of the scatter from window `cw` into the layout `nx` (see
// TcWin::rotm): the 16 lanes of a half-warp hold rows whose bits 0-3 are the
// lane bits; the rotation that makes their bank pairs distinct at every step,
// else the one with the fewest repeats.
static uint16_t tc_rotation(const TcWin &cw, const TcWin &nx) {
    uint32_t rowc[4], winc[3];
    for (int t = 0; t < 4; ++t) rowc[t] = nx.cb[cw.row[t]];
    for (int q = 0; q < 3; ++q) winc[q] = nx.cb[cw.win[q]];
    int best = 1 << 30;
    uint16_t best_m = 0;
    for (uint32_t m = 0; m < (1u << 12); ++m) {
        int cost = 0;
        for (int step = 0; step < 8 && cost < best; ++step) {
            int hits[16] = {0}, worst = 0;
            for (int lane = 0; lane < 16; ++lane) {
                uint32_t a = 0;
                for (int t = 0; t < 4; ++t)
                    if ((lane >> t) & 1) a ^= rowc[t];
                int rot = 0;
                for (int i = 0; i < 3; ++i) rot |= (__builtin_popcount(lane & ((m >> (4 * i)) & 15u)) & 1) << i;
                const int u = step ^ rot;
                for (int q = 0; q < 3; ++q)
                    if ((u >> q) & 1) a ^= winc[q];
                worst = std::max(worst, ++hits[bank8(a)]);
            }
            cost += worst;
        }
        if (cost < best) { best = cost; best_m = (uint16_t)m; }
        if (best == 8) break;   // one wavefront per step: conflict-free
    }
    return best_m;
}

// Rank over GF(2) of 4-bit vectors.
static int rank_bits4(uint32_t *v, int nv) {
    int r = 0;
    for (int bit = 3; bit >= 0 && r < nv; --bit) {
        int p = -1;
        for (int i = r; i < nv; ++i)
            if ((v[i] >> bit) & 1u) { p = i; break; }
        if (p < 0) continue;
        std::swap(v[r], v[p]);
        for (int i = 0; i < nv; ++i)
            if (i != r && ((v[i] >> bit) & 1u)) v[i] ^= v[r];
        ++r;
    }
    return r;
}

// A window's operand layout for a given row order (tile bits of row positions 0..6).
static void tc_layout(TcWin &t, const RegPass &rp, const uint8_t *rows) {
    std::memset(&t, 0, sizeof t);
    for (int k = 0; k < kMaxWin; ++k) {
        t.win[k] = rp.win[k];
        t.cb[rp.win[k]] = tc_addr(0, 1u << k);
    }
    for (int r = 0; r < kTcRows; ++r) {
        t.row[r] = rows[r];
        t.cb[rows[r]] = tc_addr(1u << r, 0);
    }
}

// The exchange map into a window: u = the 4 tile bits the storing lanes
// differ in (bank bits 0-3 in that order), v = the loading lanes' 4 bits (the
// window's row positions 0-3).  v's bits outside u take the bank bits u's
// members among them leave free, so both sets reach all 16 bank pairs; the
// tile bits outside u give the high address bits, which makes the map a
// bijection onto the 4096 8-byte slots.
static void tc_exchange(uint32_t *xcb, const uint8_t *u, const uint8_t *v) {
    uint32_t g[kTcTile] = {0};
    bool in_u[kTcTile] = {false};
    for (int i = 0; i < 4; ++i) {
        g[u[i]] = 1u << i;
        in_u[u[i]] = true;
    }
    uint32_t covered = 0;
    for (int i = 0; i < 4; ++i)
        if (in_u[v[i]]) covered |= g[v[i]];
    int next = 0;
    for (int i = 0; i < 4; ++i)
        if (!in_u[v[i]]) {
            while ((covered >> next) & 1u) ++next;
            g[v[i]] = 1u << next;
            covered |= 1u << next;
        }
    for (int b = 0, h = 0; b < kTcTile; ++b) {
        xcb[b] = g[b] << 3;
        if (!in_u[b]) xcb[b] |= 1u << (7 + h++);
    }
}

std::vector<TcWin> make_tc_windows(const BrickHostPlan &P) {
    std::vector<TcWin> out(P.rpasses.size());
    for (const BrickPass &ps : P.passes) {
        // Row orders of the pass's windows.  The 16 lanes of a half-warp drain the
        // rows that differ in row positions 0-3 and store into the next window's
        // layout; they hit distinct 8-byte bank pairs when those 4 tile bits have
        // linearly independent bank contributions there (next-window positions 0-3:
        // bank bits 0-3; next-layout row positions 0, 1, 2: bank bits 1, 2, 3 through
        // the swizzle; the rest: none).  A dynamic program over the ordered choice
        // of the first 4 row positions of every window minimises the rank deficit
        // summed over the transitions; the rest of the rows stay ascending.
        const int nw = ps.n_rp;
        std::vector<std::vector<uint8_t>> rowbits(nw);
        for (int w = 0; w < nw; ++w) {
            const RegPass &rp = P.rpasses[ps.rp_off + w];
            int in_win[32] = {0};
            for (int k = 0; k < kMaxWin; ++k) in_win[rp.win[k]] = 1;
            for (int b = 0; b < kTcTile; ++b)
                if (!in_win[b]) rowbits[w].push_back((uint8_t)b);
        }
        // candidate prefixes: ordered 4-tuples of distinct row bits (indices into rowbits)
        std::vector<std::array<uint8_t, 4>> pre;
        for (int a = 0; a < kTcRows; ++a)
            for (int b = 0; b < kTcRows; ++b)
                for (int c = 0; c < kTcRows; ++c)
                    for (int d = 0; d < kTcRows; ++d)
                        if (a != b && a != c && a != d && b != c && b != d && c != d)
                            pre.push_back({(uint8_t)a, (uint8_t)b, (uint8_t)c, (uint8_t)d});
        const int np = (int)pre.size();
        auto rows_of = [&](int w, int pi, uint8_t *rows) {
            bool used[kTcRows] = {false};
            for (int i = 0; i < 4; ++i) {
                rows[i] = rowbits[w][pre[pi][i]];
                used[pre[pi][i]] = true;
            }
            for (int j = 0, r = 4; j < kTcRows; ++j)
                if (!used[j]) rows[r++] = rowbits[w][j];
        };
        // bank contribution (4 bits) of tile bit b in window w's layout with prefix pi
        auto bank = [&](int w, int pi, int b) -> uint32_t {
            const RegPass &rp = P.rpasses[ps.rp_off + w];
            for (int k = 0; k < kMaxWin; ++k)
                if (rp.win[k] == b) return k < 4 ? 1u << k : 0u;
            for (int r = 0; r < 3; ++r)
                if (rowbits[w][pre[pi][r]] == b) return 1u << (r + 1);
            return 0u;
        };
        std::vector<std::vector<int>> cost(nw, std::vector<int>(np, 0)), from(nw, std::vector<int>(np, -1));
        std::vector<uint32_t> bk((size_t)np * kTcTile);
        for (int w = 1; w < nw; ++w) {
            for (int q = 0; q < np; ++q)
                for (int b = 0; b < kTcTile; ++b) bk[(size_t)q * kTcTile + b] = bank(w, q, b);
            // the transition depends on the previous prefix only through its 4 lane bits
            for (int q = 0; q < np; ++q) {
                int best = 1 << 30, arg = 0;
                const uint32_t *bq = &bk[(size_t)q * kTcTile];
                for (int p = 0; p < np && best > 0; ++p) {
                    if (cost[w - 1][p] >= best) continue;
                    uint32_t v[4];
                    for (int i = 0; i < 4; ++i) v[i] = bq[rowbits[w - 1][pre[p][i]]];
                    const int c = cost[w - 1][p] + 4 - rank_bits4(v, 4);
                    if (c < best) { best = c; arg = p; }
                }
                cost[w][q] = best;
                from[w][q] = arg;
            }
        }
        int q = 0;
        for (int i = 1; i < np; ++i)
            if (cost[nw - 1][i] < cost[nw - 1][q]) q = i;
        std::vector<int> choice(nw);
        for (int w = nw - 1; w >= 0; --w) {
            choice[w] = q;
            if (w > 0) q = from[w][q];
        }
        for (int w = 0; w < nw; ++w) {
            uint8_t rows[kTcRows];
            rows_of(w, choice[w], rows);
            tc_layout(out[ps.rp_off + w], P.rpasses[ps.rp_off + w], rows);
        }
        for (int w = 0; w + 1 < nw; ++w) out[ps.rp_off + w].rotm = tc_rotation(out[ps.rp_off + w], out[ps.rp_off + w + 1]);
        const uint8_t first[4] = {0, 1, 2, 3};   // the tile load: lanes store consecutive tile indices
        for (int w = 0; w < nw; ++w)
            tc_exchange(out[ps.rp_off + w].xcb, w ? out[ps.rp_off + w - 1].row : first, out[ps.rp_off + w].row);
    }
    return out;
}

std::vector<TcXa> make_tc_xaddr(const BrickHostPlan &P, const std::vector<TcWin> &W) {
    std::vector<TcXa> out(P.rpasses.size());
    for (const BrickPass &ps : P.passes)
        for (int w = 0; w < ps.n_rp; ++w) {
            const TcWin &cw = W[ps.rp_off + w];
            TcXa &x = out[ps.rp_off + w];
            std::memset(&x, 0, sizeof x);
            const bool last = w + 1 == ps.n_rp;
            const uint32_t *lm = cw.xcb, *sm = last ? nullptr : W[ps.rp_off + w + 1].xcb;
            for (int l = 0; l < 32; ++l)
                for (int t = 0; t < 5; ++t)
                    if ((l >> t) & 1) {
                        x.ld_lane[l] ^= lm[cw.row[t]];
                        if (sm) x.st_lane[l] ^= sm[cw.row[t]];
                    }
            for (int wp = 0; wp < 8; ++wp) {
                for (int t = 5; t < kTcRows; ++t)
                    if (((wp & 3) >> (t - 5)) & 1) {
                        x.ld_warp[wp] ^= lm[cw.row[t]];
                        if (sm) x.st_warp[wp] ^= sm[cw.row[t]];
                    }
                if (wp >> 2) {
                    x.ld_warp[wp] ^= lm[cw.win[4]];
                    if (sm) x.st_warp[wp] ^= sm[cw.win[4]];
                }
            }
            for (int k = 0; k < 4; ++k) {
                x.ld_c[k] = lm[cw.win[k]];
                if (sm) x.st_c[k] = sm[cw.win[k]];
            }
        }
    return out;
}

}  // namespace fpk
