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

}  // namespace

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
