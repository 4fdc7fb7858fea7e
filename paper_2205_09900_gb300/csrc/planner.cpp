// planner.cpp -- contraction planner for Tr(U^dagger V) on an open chain.
//
// The trace of a circuit is the closed tensor network whose wires are joined
// output-to-input on every qubit (paper: Sec. "Algorithm description", Fig. 3a)
// and it is contracted along the qubit (space) direction so that the number of
// exposed indices stays minimal (same section).  Here:
//   1. U^dagger V is written as the cyclic operator sequence V's gates (first
//      to last) followed by U's gates (last to first, conjugate-transposed).
//   2. Operators with the same support that meet once everything in between
//      has commuted out of the way are multiplied together ("merged"): the
//      last layers of U and V, the first layers (cyclically), and CZ pairs,
//      which cancel.  For brickwork this leaves l-1 gates per bond.
//   3. Every qubit's wire is cut into segments by its non-diagonal operators;
//      a segment is a binary variable, an operator is a factor over the
//      segments it touches (diagonal operators do not cut the wire).
//   4. The variables are summed out site by site from both chain ends towards
//      bond `cut`; each factor becomes one sweep operation that multiplies the
//      boundary by a <=16-entry table and sums the variables it is the last
//      factor of.  The two boundaries meet in a dot product.
// For brickwork every interior operation is an in-place 4x4 map on two
// boundary bits: the boundary is a state over the 2(l-1) segments of one
// qubit, and the sweep is a brickwork circuit in the space direction.
#include "planner.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>

namespace fpk {

std::vector<GateSlot> layout_brickwork(int n, int l) {
    std::vector<GateSlot> g;
    int raw = 0;
    for (int t = 1; t <= l; ++t)
        for (int b = (t - 1) % 2; b <= n - 2; b += 2) g.push_back({0, b, raw++});
    return g;
}

std::vector<GateSlot> layout_hea(int n, int L) {
    std::vector<GateSlot> g;
    for (int t = 0; t < L; ++t) {
        for (int q = 0; q < n; ++q) g.push_back({1, q, t * n + q});
        for (int b = 0; b <= n - 2; ++b) g.push_back({2, b, -1});
    }
    return g;
}

std::vector<GateSlot> layout_hea_pauli(int n, int L, bool cz) {
    std::vector<GateSlot> g;
    for (int q = 0; q < n; ++q) g.push_back({1, q, 1 + q});   // RY(pi/4) wall
    for (int t = 0; t < L; ++t) {
        for (int q = 0; q < n; ++q) g.push_back({1, q, 1 + n + t * n + q});
        for (int par = 0; par < 2; ++par)
            for (int b = par; b <= n - 2; b += 2) {
                if (!cz) g.push_back({3, b + 1, 0});          // H on the target
                g.push_back({2, b, -1});
                if (!cz) g.push_back({3, b + 1, 0});
            }
    }
    return g;
}

std::vector<GateSlot> layout_local(int n, const std::vector<int> &bonds) {
    (void)n;
    std::vector<GateSlot> g;
    for (size_t i = 0; i < bonds.size(); ++i) g.push_back({0, bonds[i], (int)i});
    return g;
}

namespace {

struct SeqEl {
    int kind;                       // 0 gate2 (data), 1 gate1 (data), 2 constant diagonal
    int q;
    bool invol = false;             // a lone constant involution (GateSlot kind 3)
    std::vector<MergeRef> chain;    // application order
    double dre[4], dim[4];          // kind 2 entries
};

bool overlaps(const SeqEl &a, const SeqEl &b) {
    int a0 = a.q, a1 = a.kind == 1 ? a.q : a.q + 1;
    int b0 = b.q, b1 = b.kind == 1 ? b.q : b.q + 1;
    return !(a1 < b0 || b1 < a0);
}

bool commute(const SeqEl &a, const SeqEl &b) {
    if (!overlaps(a, b)) return true;
    return a.kind == 2 && b.kind == 2;   // diagonal operators commute
}

bool same_support(const SeqEl &a, const SeqEl &b) { return a.kind == b.kind && a.q == b.q; }

void merge_sequence(std::vector<SeqEl> &seq) {
    // The sequence is cyclic; merged-away operators are unlinked from a
    // doubly linked ring (no element moves), and passes in index order repeat
    // until nothing merges.  Survivors keep their relative order.
    const int N0 = (int)seq.size();
    if (N0 < 2) return;
    std::vector<int> nxt(N0), prv(N0);
    std::vector<char> alive(N0, 1);
    for (int i = 0; i < N0; ++i) {
        nxt[i] = (i + 1) % N0;
        prv[i] = (i + N0 - 1) % N0;
    }
    int n_alive = N0;
    auto unlink = [&](int i) {
        nxt[prv[i]] = nxt[i];
        prv[nxt[i]] = prv[i];
        alive[i] = 0;
        --n_alive;
    };
    bool changed = true;
    while (changed && n_alive > 1) {
        changed = false;
        for (int i = 0; i < N0 && n_alive > 1; ++i) {
            if (!alive[i]) continue;
            // walk forward (cyclically) while seq[i] commutes with what it passes;
            // stop at the first operator with the same support (merge) or the
            // first one it does not commute with (no merge)
            int j = -1;
            for (int s = 1, k = nxt[i]; s < n_alive; ++s, k = nxt[k]) {
                if (same_support(seq[i], seq[k])) { j = k; break; }
                if (!commute(seq[i], seq[k])) break;
            }
            if (j < 0) continue;
            // seq[i] moves forward (cyclically) past commuting operators to seq[j]
            SeqEl &m = seq[j];
            if (m.kind == 2) {
                bool ident = true;
                for (int e = 0; e < 4; ++e) {
                    double re = seq[i].dre[e] * m.dre[e] - seq[i].dim[e] * m.dim[e];
                    double im = seq[i].dre[e] * m.dim[e] + seq[i].dim[e] * m.dre[e];
                    m.dre[e] = re; m.dim[e] = im;
                    if (re != 1.0 || im != 0.0) ident = false;
                }
                if (ident) unlink(j);   // CZ . CZ = identity: both go
            } else if (seq[i].invol && m.invol && seq[i].chain[0].gate == m.chain[0].gate) {
                unlink(j);   // H . H = identity: both go
            } else {
                // application order: seq[i]'s chain first, then m's
                m.invol = false;
                std::vector<MergeRef> c = std::move(seq[i].chain);
                c.insert(c.end(), m.chain.begin(), m.chain.end());
                m.chain = std::move(c);
            }
            unlink(i);
            changed = true;
        }
    }
    std::vector<SeqEl> out;
    out.reserve(n_alive);
    for (int i = 0; i < N0; ++i)
        if (alive[i]) out.push_back(std::move(seq[i]));
    seq = std::move(out);
}

struct Factor {
    int kind;               // 0 gate2, 1 gate1, 2 const diag, 3 gate1 times a +-1 diagonal
    int q;
    int merged;             // merged gate id (kinds 0, 1, 3)
    int slot_var[4];        // gate2: out_q, out_q1, in_q, in_q1; gate1: out, in; diag: y_q, y_q1;
                            // kind 3: gate1's out, in, then the diagonal's y_q, y_q1
    int nslots;
    double dre[4], dim[4];
    int side;               // 0 left, 1 right
    int site;
};

int slot_entry(const Factor &f, const int *val) {
    if (f.kind == 0) return (val[0] * 2 + val[1]) * 4 + (val[2] * 2 + val[3]);
    if (f.kind == 1 || f.kind == 3) return val[0] * 2 + val[1];
    return val[0] * 2 + val[1];   // diagonal index
}

bool shares_var(const Factor &a, const Factor &b) {
    for (int i = 0; i < a.nslots; ++i)
        for (int j = 0; j < b.nslots; ++j)
            if (a.slot_var[i] == b.slot_var[j]) return true;
    return false;
}

bool sign_diagonal(const Factor &f) {   // a constant diagonal with entries +-1 (CZ products)
    for (int e = 0; e < 4; ++e)
        if (f.dim[e] != 0.0 || (f.dre[e] != 1.0 && f.dre[e] != -1.0)) return false;
    return true;
}

// cyclic sequence of U^dagger V (V's gates first to last, then U's last to
// first, conjugate-transposed), merged
std::vector<SeqEl> merged_cycle(const std::vector<GateSlot> &U, const std::vector<GateSlot> &V, int raw_kind) {
    const int dim = raw_kind == RAW_ROT2 ? 2 : 4;
    std::vector<SeqEl> seq;
    auto push = [&](const GateSlot &g, int which, int dagger) {
        SeqEl e;
        e.kind = g.kind == 3 ? 1 : g.kind;
        e.invol = g.kind == 3;
        e.q = g.q;
        for (int k = 0; k < 4; ++k) { e.dre[k] = 1; e.dim[k] = 0; }
        if (g.kind == 2) {
            e.dre[3] = -1.0;   // CZ = diag(1, 1, 1, -1), its own conjugate
        } else {
            e.chain.push_back({which, g.raw, dagger, e.kind == 1 ? 2 : dim});
        }
        seq.push_back(e);
    };
    for (const auto &g : V) push(g, 1, 0);
    for (auto it = U.rbegin(); it != U.rend(); ++it) push(*it, 0, 1);
    merge_sequence(seq);
    return seq;
}

}  // namespace

// Spiral program.  Every wire of the merged cycle is cut by its 1-qubit
// operators into segments; a CZ on bond (q, q+1) couples one segment of q and
// one of q+1 with (-1)^{y y'} = H[y][y'] (H = [[1, 1], [1, -1]]).  When every
// segment of a wire holds exactly one CZ, qubit q is a ring of segments tapped
// on the left (L) or the right (R) bond, consecutive segments joined by the
// 1-qubit operators X[out][in].  The state holds one variable per CZ of a bond
// (the neighbouring qubit's segment, before the CZ coupling H) plus an
// auxiliary bit; qubit q turns it into the variables of its R segments:
// START couples the ring's first L segment S_0 (H), sums the old auxiliary
// bit and copies S_0 into it; then the ring is walked S_0, S_1, ... back to
// S_0 (reached through the auxiliary copy), one 4x4 map per step:
//   L -> R   the R segment takes the L segment's bit (fused with the next step);
//   R -> L   the L bit is coupled (H) and multiplied by X (the R bit stays);
//   L -> L   the old L is summed out and its bit zeroed (freed);
//   R -> R   the new R takes a freed bit.
// The walk starts at an L segment from which every R -> R step finds a freed
// bit (L -> L and R -> R steps are equally many on a ring with as many L as R
// segments).  The first qubit (R taps only) starts from delta(aux, S_0's bit)
// and multiplies X[S_{i+1}][S_i] on its ring; the last (L taps only) couples
// and multiplies without freeing; the trace is the sum of the final state.
// Map entries, with o/i the output/input values of bits a (low) and b (high),
// are listed at SpiralType.
SpiralPlan make_spiral_plan(int n, const std::vector<GateSlot> &U, const std::vector<GateSlot> &V, int raw_kind) {
    SpiralPlan P;
    std::vector<SeqEl> seq = merged_cycle(U, V, raw_kind);
    std::vector<int> item(seq.size(), -1), tap(seq.size(), -1), ntap(n, 0);
    for (size_t i = 0; i < seq.size(); ++i) {
        const SeqEl &e = seq[i];
        if (e.kind == 0) { P.why = "two-qubit gates"; return P; }
        if (e.kind == 2) {
            for (int k = 0; k < 4; ++k)
                if (e.dim[k] != 0.0 || e.dre[k] != (k == 3 ? -1.0 : 1.0)) { P.why = "diagonal other than CZ"; return P; }
            tap[i] = ntap[e.q]++;
            continue;
        }
        item[i] = (int)P.merges.size();
        MergeItem mi;
        mi.first = (int)P.refs.size();
        mi.count = (int)e.chain.size();
        P.refs.insert(P.refs.end(), e.chain.begin(), e.chain.end());
        P.merges.push_back(mi);
    }
    const int M = n >= 2 ? ntap[0] : 0;
    if (n < 3 || M < 1) { P.why = "no CZ left"; return P; }
    for (int b = 0; b < n - 1; ++b)
        if (ntap[b] != M) { P.why = "bonds with different CZ counts"; return P; }
    if (M + 1 > FP_MAX_STATE_BITS) { P.why = "boundary too large"; return P; }
    P.bits = M + 1;
    const int aux = M;
    std::vector<int> pos(M);   // state bit of each CZ of the current bond
    auto map = [&](int a, int b, int type, int f, int g) {
        P.maps.push_back({(uint8_t)a, (uint8_t)b, (uint8_t)type, 0, f, g});
    };
    for (int q = 0; q < n; ++q) {
        // the wire of q in cyclic order: 1-qubit items and taps (side 0 left, 1 right)
        struct Ev { int op, side, id; };
        std::vector<Ev> ev;
        for (size_t i = 0; i < seq.size(); ++i) {
            const SeqEl &e = seq[i];
            if (e.kind == 1 && e.q == q) ev.push_back({item[i], -1, -1});
            else if (e.kind == 2 && e.q == q - 1) ev.push_back({-1, 0, tap[i]});
            else if (e.kind == 2 && e.q == q) ev.push_back({-1, 1, tap[i]});
        }
        int first_op = -1;
        for (size_t i = 0; i < ev.size(); ++i) if (ev[i].op >= 0) { first_op = (int)i; break; }
        if (first_op < 0) { P.why = "a wire without 1-qubit operators"; return P; }
        struct Seg { int side, id, op_out; };   // op_out: the operator leaving the segment
        std::vector<Seg> segs;
        const int E = (int)ev.size();
        for (int k = 0; k < E; ++k) {
            if (ev[(first_op + k) % E].op < 0) continue;
            int side = -1, id = -1, cnt = 0, j = 1;
            for (; j < E; ++j) {
                const Ev &y = ev[(first_op + k + j) % E];
                if (y.op >= 0) break;
                side = y.side; id = y.id; ++cnt;
            }
            if (cnt != 1) { P.why = "a segment without exactly one CZ"; return P; }
            segs.push_back({side, id, ev[(first_op + k + j) % E].op});
        }
        const int S = (int)segs.size();
        const bool first = q == 0, last = q == n - 1;
        if ((first || last) ? S != M : S != 2 * M) { P.why = "segment count"; return P; }
        if (first) {
            for (int i = 0; i < M; ++i) {
                if (segs[i].side != 1) { P.why = "left taps on the first qubit"; return P; }
                pos[segs[i].id] = i;
            }
            P.first_bit = pos[segs[0].id];
            for (int i = 0; i < M; ++i)
                map(pos[segs[i].id], i + 1 < M ? pos[segs[i + 1].id] : aux, SP_DIAG_BA, -1, segs[i].op_out);
            continue;
        }
        if (last) {
            for (int i = 0; i < M; ++i)
                if (segs[i].side != 0) { P.why = "right taps on the last qubit"; return P; }
            map(aux, pos[segs[0].id], SP_START, -1, -1);
            for (int i = 0; i + 1 < M; ++i) map(pos[segs[i].id], pos[segs[i + 1].id], SP_RL, -1, segs[i].op_out);
            map(pos[segs[M - 1].id], aux, SP_DIAG_BA, -1, segs[M - 1].op_out);
            continue;
        }
        // start: an L segment from which freed bits always precede their use
        int s0 = -1;
        for (int c = 0; c < S && s0 < 0; ++c) {
            if (segs[c].side != 0) continue;
            int bal = 0;
            bool ok = true;
            for (int k = 0; k < S && ok; ++k) {
                const int a = segs[(c + k) % S].side, b = segs[(c + k + 1) % S].side;
                if (a == 0 && b == 0) ++bal;
                if (a == 1 && b == 1 && --bal < 0) ok = false;
            }
            if (ok) s0 = c;
        }
        if (s0 < 0) { P.why = "no valid start on the ring"; return P; }
        std::vector<int> npos(M, -1), freed;
        map(aux, pos[segs[s0].id], SP_START, -1, -1);
        int cb = pos[segs[s0].id], cside = 0, pendF = -1;   // carry bit, its side, deferred L -> R operator
        for (int k = 0; k < S; ++k) {
            const Seg &cur = segs[(s0 + k) % S];
            const bool close = k == S - 1;                  // the step back to S_0 (through aux)
            const Seg &nxt = segs[(s0 + k + 1) % S];
            const int op = cur.op_out;
            const int nb = close ? aux : pos[nxt.id];
            if (cside == 0 && nxt.side == 1) {              // L -> R: deferred
                if (close) { P.why = "ring closes on R"; return P; }
                pendF = op;
                cside = 1;
                npos[nxt.id] = cb;
                continue;
            }
            if (cside == 0 && nxt.side == 0) {              // L -> L: free the carry's bit
                map(cb, nb, close ? SP_LL_AUX : SP_LL, -1, op);
                freed.push_back(cb);
                cb = nb;
                continue;
            }
            if (nxt.side == 0) {                            // R -> L
                if (pendF >= 0) map(cb, nb, close ? SP_MID_AUX : SP_MID, pendF, op);
                else if (close) map(cb, nb, SP_DIAG_BA, -1, op);
                else map(cb, nb, SP_RL, -1, op);
                pendF = -1;
                cside = 0;
                cb = nb;
                continue;
            }
            // R -> R: the new R segment takes a freed bit
            if (freed.empty()) { P.why = "no freed bit"; return P; }
            const int fb = freed.back();
            freed.pop_back();
            if (pendF >= 0) map(cb, fb, SP_MID_RR, pendF, op);
            else map(cb, fb, SP_RR, -1, op);
            pendF = -1;
            npos[nxt.id] = fb;
            cb = fb;
        }
        for (int u = 0; u < M; ++u)
            if (npos[u] < 0) { P.why = "an R segment without a bit"; return P; }
        pos = npos;
    }
    P.ok = true;
    return P;
}

static uint32_t spiral_swizzle(uint32_t y) {   // s(y) of the spiral window kernel
    const uint32_t q = y >> 4;
    return y ^ ((q ^ (q >> 4) ^ (q >> 8) ^ (q >> 12)) & 15u);
}

void spiral_windows(const SpiralPlan &P, int R, int split, std::vector<SpiralWin> &wins, std::vector<uint8_t> &ij,
                    int h_out[2]) {
    wins.clear();
    ij.assign(P.maps.size(), 0);
    R = std::min(std::max(R, 2), std::min(kSpiralMaxWin, P.bits));
    // runs of consecutive maps on at most R bits
    std::vector<uint32_t> sets;
    std::vector<std::pair<size_t, size_t>> runs;
    for (size_t k = 0; k < P.maps.size();) {
        uint32_t set = 0;
        size_t e = k;
        for (; e < P.maps.size(); ++e) {
            const uint32_t s2 = set | (1u << P.maps[e].a) | (1u << P.maps[e].b);
            if (__builtin_popcount(s2) > R || e - k >= (size_t)kSpiralWinMaxMaps) break;
            set = s2;
        }
        sets.push_back(set);
        runs.push_back({k, e});
        k = e;
    }
    // cluster bits: the state bits the fewest runs touch
    int hb[2] = {-1, -1};
    {
        std::vector<std::pair<int, int>> use;   // (runs touching the bit, bit)
        for (int b = 0; b < P.bits; ++b) {
            int c = 0;
            for (uint32_t s : sets) c += (s >> b) & 1;
            use.push_back({c, b});
        }
        std::sort(use.begin(), use.end());
        for (int q = 0; q < split && q < 2; ++q) hb[q] = use[q].second;
        if (split == 2 && hb[0] > hb[1]) std::swap(hb[0], hb[1]);
    }
    uint32_t hmask = 0;
    for (int q = 0; q < 2; ++q) if (hb[q] >= 0) hmask |= 1u << hb[q];
    for (size_t i = 0; i < runs.size(); ++i) {
        // pad to R bits with the lowest other non-cluster bits (every window moves 2^R amplitudes)
        uint32_t &set = sets[i];
        for (int pass = 0; pass < 2; ++pass)
            for (int b = 0; b < P.bits && __builtin_popcount(set) < R; ++b)
                if (pass == 1 || !(hmask >> b & 1)) set |= 1u << b;
        SpiralWin w;
        std::memset(&w, 0, sizeof w);
        int loc[32], nb = 0;
        for (int b = 0; b < P.bits; ++b)
            if (set & (1u << b)) { loc[b] = nb; w.bits[nb++] = (uint8_t)b; }
        w.nb = (uint8_t)nb;
        w.n_maps = (uint8_t)(runs[i].second - runs[i].first);
        w.first = (int32_t)runs[i].first;
        for (size_t m = runs[i].first; m < runs[i].second; ++m)
            ij[m] = (uint8_t)(loc[P.maps[m].a] | (loc[P.maps[m].b] << 4));
        wins.push_back(w);
    }
    if (h_out) { h_out[0] = hb[0]; h_out[1] = hb[1]; }
    auto local = [&](int b) { return b - __builtin_popcount(hmask & ((1u << b) - 1u)); };
    for (size_t i = 0; i < wins.size(); ++i) {
        SpiralWin &w = wins[i];
        const uint32_t set = sets[i];
        w.cross = (set & hmask) ? 1 : 0;
        for (int q = 0; q < w.nb; ++q) {
            const int b = w.bits[q];
            w.ctab[q] = (uint8_t)((b == hb[0] ? 1 : 0) | (b == hb[1] ? 2 : 0));
            w.off[q] = (hmask >> b & 1) ? 0 : (uint16_t)spiral_swizzle(1u << local(b));
        }
        // lane q: the free non-cluster bit of lowest local position with residue q mod 4
        // (16 lanes then touch 16 distinct slots of sw), else the lowest one left
        const uint32_t freem = ((1u << P.bits) - 1u) & ~set;
        uint32_t lanes = 0;
        int n = 0;
        for (int q = 0; q < 4; ++q) {
            int pick = -1;
            for (int b = 0; b < P.bits && pick < 0; ++b)
                if ((freem & ~hmask & ~lanes) >> b & 1 && local(b) % 4 == q) pick = b;
            for (int b = 0; b < P.bits && pick < 0; ++b)
                if ((freem & ~hmask & ~lanes) >> b & 1) pick = b;
            if (pick >= 0) { lanes |= 1u << pick; w.pos[n++] = (uint8_t)pick; }
        }
        for (int b = 0; b < P.bits; ++b)
            if ((freem & ~hmask & ~lanes) >> b & 1) w.pos[n++] = (uint8_t)b;
        for (int b = 0; b < P.bits; ++b)
            if ((freem & hmask) >> b & 1) w.pos[n++] = (uint8_t)b;
        w.n_pos = (uint8_t)n;
    }
}

HostPlan make_plan(int n, const std::vector<GateSlot> &U, const std::vector<GateSlot> &V,
                   int raw_kind, int n_raw, int cut, int max_bits) {
    HostPlan P;
    max_bits = std::min(max_bits, FP_MAX_STATE_BITS);   // device tables are sized for this
    P.n = n;
    P.n_raw = n_raw;
    P.raw_kind = raw_kind;
    const int dim = raw_kind == RAW_ROT2 ? 2 : 4;

    // 1. cyclic sequence of U^dagger V
    std::vector<SeqEl> seq;
    auto push = [&](const GateSlot &g, int which, int dagger) {
        SeqEl e;
        e.kind = g.kind == 3 ? 1 : g.kind;
        e.invol = g.kind == 3;
        e.q = g.q;
        for (int k = 0; k < 4; ++k) { e.dre[k] = 1; e.dim[k] = 0; }
        if (g.kind == 2) {
            e.dre[3] = -1.0;   // CZ = diag(1, 1, 1, -1), its own conjugate
        } else {
            e.chain.push_back({which, g.raw, dagger, e.kind == 1 ? 2 : dim});
        }
        seq.push_back(e);
    };
    for (const auto &g : V) push(g, 1, 0);
    for (auto it = U.rbegin(); it != U.rend(); ++it) push(*it, 0, 1);

    // 2. merges
    merge_sequence(seq);
    for (auto &e : seq) {
        if (e.kind == 2) continue;
        MergeItem mi;
        mi.first = (int)P.refs.size();
        mi.count = (int)e.chain.size();
        P.refs.insert(P.refs.end(), e.chain.begin(), e.chain.end());
        P.merges.push_back(mi);
    }

    // 3. segments and factors
    std::vector<int> s(n, 0), base(n + 1, 0);
    std::vector<std::vector<int>> posq(seq.size());
    for (size_t t = 0; t < seq.size(); ++t) {
        const SeqEl &e = seq[t];
        int nq = e.kind == 1 ? 1 : 2;
        for (int i = 0; i < nq; ++i) {
            int q = e.q + i;
            if (e.kind == 2) posq[t].push_back(s[q] - 1);
            else posq[t].push_back(s[q]++);
        }
    }
    for (int q = 0; q < n; ++q) base[q + 1] = base[q] + std::max(s[q], 1);
    const int nvars = base[n];
    std::vector<Factor> fs;
    int merged_id = 0;
    for (size_t t = 0; t < seq.size(); ++t) {
        const SeqEl &e = seq[t];
        Factor f;
        f.kind = e.kind;
        f.q = e.q;
        f.merged = e.kind == 2 ? -1 : merged_id++;
        for (int k = 0; k < 4; ++k) { f.dre[k] = e.dre[k]; f.dim[k] = e.dim[k]; }
        int nq = e.kind == 1 ? 1 : 2, sin[2], sout[2];
        for (int i = 0; i < nq; ++i) {
            int q = e.q + i, sq = std::max(s[q], 1), j = posq[t][i];
            if (e.kind == 2) {
                int cur = j >= 0 ? j : sq - 1;
                sin[i] = sout[i] = base[q] + cur;
            } else {
                sout[i] = base[q] + j;
                sin[i] = base[q] + (j - 1 + sq) % sq;
            }
        }
        if (e.kind == 0) {
            f.slot_var[0] = sout[0]; f.slot_var[1] = sout[1];
            f.slot_var[2] = sin[0];  f.slot_var[3] = sin[1];
            f.nslots = 4;
        } else if (e.kind == 1) {
            f.slot_var[0] = sout[0]; f.slot_var[1] = sin[0];
            f.nslots = 2;
        } else {
            f.slot_var[0] = sout[0]; f.slot_var[1] = sout[1];
            f.nslots = 2;
        }
        if (e.kind == 1) { f.side = e.q < cut ? 0 : 1; f.site = e.q; }
        else { f.side = e.q < cut ? 0 : 1; f.site = f.side == 0 ? e.q : e.q + 1; }
        fs.push_back(f);
    }

    // variable occurrence per side; free loops
    std::vector<int> nocc(nvars, 0), side_mask(nvars, 0);
    for (auto &f : fs) {
        int seen[4], ns = 0;
        for (int k = 0; k < f.nslots; ++k) {
            int v = f.slot_var[k];
            bool dup = false;
            for (int z = 0; z < ns; ++z) dup |= seen[z] == v;
            if (dup) continue;
            seen[ns++] = v;
            nocc[v]++;
            side_mask[v] |= 1 << f.side;
        }
    }
    int free_loops = 0;
    for (int v = 0; v < nvars; ++v) if (nocc[v] == 0) ++free_loops;
    P.prefactor = std::ldexp(1.0, free_loops);

    // processing orders
    std::vector<int> order[2];
    for (int side = 0; side < 2; ++side) {
        std::vector<std::pair<std::pair<int, int>, int>> key;
        for (size_t i = 0; i < fs.size(); ++i) {
            if (fs[i].side != side) continue;
            int sk = side == 0 ? fs[i].site : (n - 1 - fs[i].site);
            key.push_back({{sk, (int)i}, (int)i});
        }
        std::sort(key.begin(), key.end());
        for (auto &k : key) order[side].push_back(k.second);
    }

    // Fusion: a constant +-1 diagonal (CZ) next to a 1-qubit factor on a shared
    // segment in the processing order becomes one factor over their <= 3 segments.
    // The CZ otherwise opens the neighbour's segment while the shared segment is
    // still waiting for the 1-qubit op that closes it, one boundary bit more.
    for (int side = 0; side < 2; ++side) {
        std::vector<int> fused;
        const std::vector<int> &ord = order[side];
        for (size_t p = 0; p < ord.size(); ++p) {
            if (p + 1 < ord.size()) {
                const Factor A = fs[ord[p]], B = fs[ord[p + 1]];
                const bool ab = A.kind == 2 && B.kind == 1, ba = A.kind == 1 && B.kind == 2;
                if ((ab || ba) && shares_var(A, B)) {
                    const Factor &X = ab ? B : A, &D = ab ? A : B;
                    if (sign_diagonal(D)) {
                        Factor F = X;
                        F.kind = 3;
                        F.slot_var[2] = D.slot_var[0];
                        F.slot_var[3] = D.slot_var[1];
                        F.nslots = 4;
                        for (int e = 0; e < 4; ++e) { F.dre[e] = D.dre[e]; F.dim[e] = 0.0; }
                        fs.push_back(F);
                        fused.push_back((int)fs.size() - 1);
                        ++p;
                        continue;
                    }
                }
            }
            fused.push_back(ord[p]);
        }
        order[side] = fused;
    }

    // 4. sweep programs
    std::vector<int> final_layout[2];
    int bits_max = 0;
    for (int side = 0; side < 2; ++side) {
        std::vector<int> last(nvars, -1);
        for (size_t p = 0; p < order[side].size(); ++p) {
            const Factor &f = fs[order[side][p]];
            for (int k = 0; k < f.nslots; ++k) last[f.slot_var[k]] = (int)p;
        }
        std::vector<int> layout;   // var at each bit position
        for (size_t p = 0; p < order[side].size(); ++p) {
            const Factor &f = fs[order[side][p]];
            int dv[4], nd = 0;
            for (int k = 0; k < f.nslots; ++k) {
                int v = f.slot_var[k];
                bool dup = false;
                for (int z = 0; z < nd; ++z) dup |= dv[z] == v;
                if (!dup) dv[nd++] = v;
            }
            std::vector<int> cons, keep, nw, sumv;
            for (int z = 0; z < nd; ++z) {
                int v = dv[z];
                bool present = std::find(layout.begin(), layout.end(), v) != layout.end();
                bool is_last = last[v] == (int)p && side_mask[v] != 3;
                if (present) (is_last ? cons : keep).push_back(v);
                else (is_last ? sumv : nw).push_back(v);
            }
            std::vector<int> cpos;
            for (int v : cons) cpos.push_back((int)(std::find(layout.begin(), layout.end(), v) - layout.begin()));
            // sort consumed by position
            std::vector<int> ci(cons.size());
            for (size_t z = 0; z < ci.size(); ++z) ci[z] = (int)z;
            std::sort(ci.begin(), ci.end(), [&](int a, int b) { return cpos[a] < cpos[b]; });
            std::vector<int> cons_s, cpos_s;
            for (int z : ci) { cons_s.push_back(cons[z]); cpos_s.push_back(cpos[z]); }
            std::vector<int> out;
            std::vector<int> npos;
            if (!cons_s.empty() && nw.size() == cons_s.size()) {
                out = layout;
                for (size_t z = 0; z < nw.size(); ++z) { out[cpos_s[z]] = nw[z]; npos.push_back(cpos_s[z]); }
            } else {
                for (int v : layout)
                    if (std::find(cons_s.begin(), cons_s.end(), v) == cons_s.end()) out.push_back(v);
                for (int v : nw) { npos.push_back((int)out.size()); out.push_back(v); }
            }
            if ((int)std::max(layout.size(), out.size()) > max_bits) {
                P.infeasible = true;
                P.error = "boundary of " + std::to_string(std::max(layout.size(), out.size())) +
                          " bits exceeds the limit of " + std::to_string(max_bits);
                return P;
            }
            bits_max = std::max<int>(bits_max, (int)std::max(layout.size(), out.size()));
            DevOp op;
            std::memset(&op, 0, sizeof op);
            op.nc = (uint8_t)cons_s.size();
            op.nk = (uint8_t)keep.size();
            op.nn = (uint8_t)nw.size();
            op.b_in = (uint8_t)layout.size();
            op.b_out = (uint8_t)out.size();
            for (size_t z = 0; z < cons_s.size(); ++z) op.cons_pos[z] = (uint8_t)cpos_s[z];
            for (size_t z = 0; z < keep.size(); ++z)
                op.keep_pos[z] = (uint8_t)(std::find(out.begin(), out.end(), keep[z]) - out.begin());
            for (size_t z = 0; z < nw.size(); ++z) op.new_pos[z] = (uint8_t)npos[z];
            op.inplace2 = (op.nc == 2 && op.nn == 2 && op.nk == 0 && op.b_in == op.b_out &&
                           op.new_pos[0] == op.cons_pos[0] && op.new_pos[1] == op.cons_pos[1]);
            // recipe
            DevRecipe r;
            std::memset(&r, 0, sizeof r);
            r.merged = f.merged;
            int nbits = op.nc + op.nk + op.nn;
            r.nent = 1 << nbits;
            for (int e = 0; e < 16; ++e)
                for (int z = 0; z < 4; ++z) { r.src[e][z] = -1; r.sgn[e][z] = 1; }
            std::vector<int> ivars;   // var of each table-index bit
            for (int v : cons_s) ivars.push_back(v);
            for (int v : keep) ivars.push_back(v);
            for (int v : nw) ivars.push_back(v);
            int nsum = (int)sumv.size();
            for (int e = 0; e < r.nent; ++e) {
                int ns = 0;
                double cre = 0, cim = 0;
                for (int sv = 0; sv < (1 << nsum); ++sv) {
                    int val[4];
                    for (int k = 0; k < f.nslots; ++k) {
                        int v = f.slot_var[k], x = -1;
                        for (int z = 0; z < nbits; ++z) if (ivars[z] == v) x = (e >> z) & 1;
                        for (int z = 0; z < nsum; ++z) if (sumv[z] == v) x = (sv >> z) & 1;
                        val[k] = x;
                    }
                    int ent = slot_entry(f, val);
                    if (f.kind == 2) { cre += f.dre[ent]; cim += f.dim[ent]; }
                    else if (f.kind == 3) {   // 2x2 slot times the diagonal's sign
                        r.sgn[e][ns] = (int8_t)f.dre[val[2] * 2 + val[3]];
                        r.src[e][ns++] = (int8_t)ent;
                    } else {
                        r.src[e][ns++] = (int8_t)ent;   // 4x4 slots 0..15, 2x2 slots 0..3
                    }
                }
                r.cre[e] = cre;
                r.cim[e] = cim;
            }
            P.ops.push_back(op);
            P.recipes.push_back(r);
            P.cost += (double)(1u << op.b_out) * (double)(1u << op.nc);
            layout = out;
        }
        final_layout[side] = layout;
        (side == 0 ? P.n_left : P.n_right) = (int)order[side].size();
    }
    if (final_layout[0].size() != final_layout[1].size()) {
        P.error = "left and right boundaries differ";
        return P;
    }
    P.bits_final = (int)final_layout[0].size();
    P.bits_max = std::max(bits_max, P.bits_final);
    P.dot_perm.assign(FP_MAX_STATE_BITS, 0);
    for (int k = 0; k < P.bits_final; ++k) {
        auto it = std::find(final_layout[1].begin(), final_layout[1].end(), final_layout[0][k]);
        if (it == final_layout[1].end()) { P.error = "boundary variable mismatch"; return P; }
        P.dot_perm[k] = (uint8_t)(it - final_layout[1].begin());
    }
    P.left_final_buf = P.n_left % 2;   // ping-pong parity: buffer 0 holds the scalar start

    // brickwork fast path: every op an in-place 4x4 on two bits, same width
    P.brick_ok = P.n_left > 0 && P.n_right > 0;
    return P;
}

}  // namespace fpk
