// spiral_plan_check.cpp -- host check of the spiral program of the paper's
// hardware-efficient ansatz (planner.cpp: make_spiral_plan), independent of
// the GPU: random 2x2 unitaries for the raw gates (the CNOTs' Hadamards exact),
// the spiral maps applied to a 2^bits state in FP64, against Tr(U^dagger V)
// of the dense 2^n matrices built gate by gate (skipped with a third argument
// "nodense"), and the register-window program (addressing of the window
// kernel emulated on the host) against the map-by-map sweep.  Prints the
// differences; exit status 1 if one exceeds 1e-12 max(|Tr|, 1).
#include "planner.h"
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <algorithm>
#include <array>
#include <cmath>
using namespace fpk;
typedef std::complex<double> cd;
struct M2 { cd m[4]; };
static M2 mul(const M2 &A, const M2 &B) { M2 C; for (int r = 0; r < 2; ++r) for (int c = 0; c < 2; ++c) C.m[2*r+c] = A.m[2*r]*B.m[c] + A.m[2*r+1]*B.m[2+c]; return C; }
int main(int argc, char **argv) {
    int n = atoi(argv[1]), L = atoi(argv[2]);
    std::mt19937_64 rng(n * 100 + L);  // random unitaries for every raw 1-qubit gate (raw 0 is the Hadamard)
    std::normal_distribution<double> N01;
    auto U = layout_hea_pauli(n, L, false), V = U;
    int n_raw = 1 + n + L * n;
    SpiralPlan P = make_spiral_plan(n, U, V, RAW_PAULI);
    if (!P.ok) { printf("n=%d L=%d not spiral: %s\n", n, L, P.why.c_str()); return 2; }
    std::vector<M2> raw[2];
    for (int w = 0; w < 2; ++w) {
        raw[w].resize(n_raw);
        double h = 1 / std::sqrt(2.0);
        raw[w][0].m[0] = h; raw[w][0].m[1] = h; raw[w][0].m[2] = h; raw[w][0].m[3] = -h;
        for (int g = 1; g < n_raw; ++g) {   // random unitary via QR-free: exp of random hermitian is overkill; use random SU(2) params
            double a = N01(rng), b = N01(rng), c = N01(rng), d = N01(rng);
            double nn = std::sqrt(a*a+b*b+c*c+d*d); a/=nn; b/=nn; c/=nn; d/=nn;
            cd ph = std::polar(1.0, N01(rng));
            raw[w][g].m[0] = cd(a, b) * ph; raw[w][g].m[1] = cd(-c, d) * ph; raw[w][g].m[2] = cd(c, d) * ph; raw[w][g].m[3] = cd(a, -b) * ph;
        }
    }
    std::vector<M2> merged(P.merges.size());
    for (size_t i = 0; i < P.merges.size(); ++i) {
        M2 Mx; Mx.m[0] = 1; Mx.m[1] = 0; Mx.m[2] = 0; Mx.m[3] = 1;
        for (int c = 0; c < P.merges[i].count; ++c) {
            const MergeRef &r = P.refs[P.merges[i].first + c];
            M2 G = raw[r.which][r.gate];
            if (r.dagger) { M2 D; D.m[0] = std::conj(G.m[0]); D.m[1] = std::conj(G.m[2]); D.m[2] = std::conj(G.m[1]); D.m[3] = std::conj(G.m[3]); G = D; }
            Mx = mul(G, Mx);
        }
        merged[i] = Mx;
    }
    const int B = P.bits, aux = B - 1;
    std::vector<cd> st((size_t)1 << B, 0.0);
    for (size_t x = 0; x < st.size(); ++x) st[x] = (((x >> aux) & 1) == ((x >> P.first_bit) & 1)) ? 1.0 : 0.0;
    const double Hm[2][2] = {{1, 1}, {1, -1}};
    std::vector<std::array<cd, 16>> Tall;
    for (const SpiralMap &mp : P.maps) {
        cd T[4][4];
        const M2 *F = mp.f >= 0 ? &merged[mp.f] : nullptr, *G = mp.g >= 0 ? &merged[mp.g] : nullptr;
        for (int o = 0; o < 4; ++o) for (int f = 0; f < 4; ++f) {
            int oa = o & 1, ob = o >> 1, ia = f & 1, ib = f >> 1;
            cd v = 0;
            auto Fm = [&](int r, int c) { return F->m[2 * r + c]; };
            auto Gm = [&](int r, int c) { return G->m[2 * r + c]; };
            switch (mp.type) {
                case SP_DIAG_BA: v = (o == f) ? Gm(ib, ia) : 0.0; break;
                case SP_START: v = (oa == ob) ? Hm[ob][ib] : 0.0; break;
                case SP_MID: v = Fm(oa, ia) * Gm(ob, oa) * Hm[ob][ib]; break;
                case SP_MID_AUX: v = (ob == ib) ? Fm(oa, ia) * Gm(ob, oa) : 0.0; break;
                case SP_RL: v = (oa == ia) ? Gm(ob, ia) * Hm[ob][ib] : 0.0; break;
                case SP_MID_RR: v = (ib == 0) ? Fm(oa, ia) * Gm(ob, oa) : 0.0; break;
                case SP_RR: v = (oa == ia && ib == 0) ? Gm(ob, ia) : 0.0; break;
                case SP_LL: v = (oa == 0) ? Gm(ob, ia) * Hm[ob][ib] : 0.0; break;
                case SP_LL_AUX: v = (oa == 0 && ob == ib) ? Gm(ib, ia) : 0.0; break;
            }
            T[o][f] = v;
        }
        std::array<cd, 16> Tf;
        for (int e = 0; e < 16; ++e) Tf[e] = T[e / 4][e % 4];
        Tall.push_back(Tf);
        std::vector<cd> nx(st.size());
        for (size_t x = 0; x < st.size(); ++x) {
            int oa = (x >> mp.a) & 1, ob = (x >> mp.b) & 1, o = oa + 2 * ob;
            size_t base = x & ~(((size_t)1 << mp.a) | ((size_t)1 << mp.b));
            cd acc = 0;
            for (int f = 0; f < 4; ++f) acc += T[o][f] * st[base | ((size_t)(f & 1) << mp.a) | ((size_t)(f >> 1) << mp.b)];
            nx[x] = acc;
        }
        st.swap(nx);
    }
    cd tr_sp = 0; for (auto v : st) tr_sp += v;
    // register windows (spiral_windows): consecutive runs covering every map once,
    // in order, each of exactly min(R, bits) ascending bits holding its maps' bits;
    // then the window kernel's addressing emulated in FP64 (group bases from the
    // deposit positions, swizzled slots, 1/2/4-CTA parts): every slot of every
    // part visited once per window, every index in bounds, a window without
    // cluster bits inside its own CTA, and the same trace as map by map
    auto swz = [](uint32_t y) { uint32_t q = y >> 4; return y ^ ((q ^ (q >> 4) ^ (q >> 8) ^ (q >> 12)) & 15u); };
    auto ins0 = [](uint32_t x, int p) { return (x & ((1u << p) - 1u)) | ((x >> p) << (p + 1)); };
    auto del = [](uint32_t x, int p) { return (x & ((1u << p) - 1u)) | ((x >> (p + 1)) << p); };
    for (int R = 4; R <= 5; ++R)
        for (int split = 0; split <= 2; ++split) {
            if (B - R - split < 4) continue;   // the kernel's precondition
            std::vector<SpiralWin> wins;
            std::vector<uint8_t> ij;
            int h[2] = {-1, -1};
            spiral_windows(P, R, split, wins, ij, h);
            size_t next = 0;
            for (const SpiralWin &w : wins) {
                bool ok = w.first == (int)next && w.n_maps > 0 && w.nb == std::min(R, B) && w.n_pos == B - w.nb;
                for (int k = 1; k < w.nb; ++k) ok = ok && w.bits[k - 1] < w.bits[k];
                for (int k = 0; k < w.nb; ++k) ok = ok && w.bits[k] < B;
                for (int m = w.first; ok && m < w.first + w.n_maps; ++m) {
                    const int i = ij[m] & 15, j = ij[m] >> 4;
                    ok = i < w.nb && j < w.nb && w.bits[i] == P.maps[m].a && w.bits[j] == P.maps[m].b;
                }
                if (!ok) { printf("n=%d L=%d: bad %d-bit window at map %d\n", n, L, R, w.first); return 1; }
                next += w.n_maps;
            }
            if (next != P.maps.size()) { printf("n=%d L=%d: %d-bit windows cover %zu of %zu maps\n", n, L, R, next, P.maps.size()); return 1; }
            const int CLt = 1 << split;
            const uint32_t SL = 1u << (B - split), G = 1u << (B - R - split);
            std::vector<std::vector<cd>> buf(CLt, std::vector<cd>(SL));
            for (int r = 0; r < CLt; ++r)
                for (uint32_t y = 0; y < SL; ++y) {
                    uint32_t x = y;
                    if (split >= 1) x = ins0(x, h[0]) | ((uint32_t)(r & 1) << h[0]);
                    if (split == 2) x = ins0(x, h[1]) | ((uint32_t)((r >> 1) & 1) << h[1]);
                    buf[r][swz(y)] = (((x >> aux) ^ (x >> P.first_bit)) & 1u) ? 0.0 : 1.0;
                }
            int ncross = 0;
            for (const SpiralWin &w : wins) {
                ncross += w.cross;
                std::vector<std::vector<char>> seen(CLt, std::vector<char>(SL, 0));
                for (int r = 0; r < CLt; ++r)
                    for (uint32_t t = 0; t < G; ++t) {
                        const uint32_t tt = r * G + t;
                        uint32_t b = 0;
                        for (int j = 0; j < w.n_pos; ++j) b |= ((tt >> j) & 1u) << w.pos[j];
                        uint32_t cb = 0, lb = b;
                        if (split == 2) { cb = ((b >> h[0]) & 1u) | (((b >> h[1]) & 1u) << 1); lb = del(del(b, h[1]), h[0]); }
                        if (split == 1) { cb = (b >> h[0]) & 1u; lb = del(b, h[0]); }
                        const uint32_t pb = swz(lb);
                        const int nv = 1 << R;
                        std::vector<cd> v(nv);
                        std::vector<uint32_t> addr(nv);
                        std::vector<int> cta(nv);
                        for (int i = 0; i < nv; ++i) {
                            uint32_t a = pb, c = cb;
                            for (int k = 0; k < R; ++k) if ((i >> k) & 1) { a ^= w.off[k]; c ^= w.ctab[k]; }
                            if (a >= SL || (int)c >= CLt || seen[c][a] || (!w.cross && (int)c != r)) {
                                printf("n=%d L=%d R=%d split=%d: slot %u of CTA %u (group of CTA %d) out of range, "
                                       "revisited or remote in a local window\n", n, L, R, split, a, c, r);
                                return 1;
                            }
                            seen[c][a] = 1;
                            addr[i] = a; cta[i] = (int)c; v[i] = buf[c][a];
                        }
                        for (int m = w.first; m < w.first + w.n_maps; ++m) {
                            const int I = ij[m] & 15, J = ij[m] >> 4;
                            for (int x = 0; x < nv; ++x) {
                                if (x & ((1 << I) | (1 << J))) continue;
                                const int id[4] = {x, x | (1 << I), x | (1 << J), x | (1 << I) | (1 << J)};
                                cd y[4];
                                for (int o = 0; o < 4; ++o) {
                                    y[o] = 0;
                                    for (int f = 0; f < 4; ++f) y[o] += Tall[m][4 * o + f] * v[id[f]];
                                }
                                for (int o = 0; o < 4; ++o) v[id[o]] = y[o];
                            }
                        }
                        for (int i = 0; i < nv; ++i) buf[cta[i]][addr[i]] = v[i];
                    }
                for (int r = 0; r < CLt; ++r)
                    for (uint32_t a = 0; a < SL; ++a)
                        if (!seen[r][a]) { printf("n=%d L=%d R=%d split=%d: slot %u of CTA %d not visited\n", n, L, R, split, a, r); return 1; }
            }
            cd tw = 0;
            for (auto &bb : buf) for (auto v : bb) tw += v;
            printf("n=%d L=%d: %zu maps in %zu windows of %d bits, split %d (h=%d,%d; %d cross): |window - direct| %.2e\n",
                   n, L, P.maps.size(), wins.size(), R, split, h[0], h[1], ncross, std::abs(tw - tr_sp));
            if (std::abs(tw - tr_sp) > 1e-12 * std::max(1.0, std::abs(tr_sp))) return 1;
        }
    if (argc > 3 && std::string(argv[3]) == "nodense") {   // sizes beyond the dense check: windows only
        printf("n=%d L=%d bits=%d maps=%zu: spiral %.12f%+.12fi (no dense check)\n", n, L, B, P.maps.size(),
               tr_sp.real(), tr_sp.imag());
        return 0;
    }
    // dense reference
    size_t D = (size_t)1 << n;
    auto build = [&](int w) {
        std::vector<cd> Mt(D * D, 0.0);
        for (size_t i = 0; i < D; ++i) Mt[i * D + i] = 1;
        for (const GateSlot &g : (w ? V : U)) {
            std::vector<cd> Nt(D * D, 0.0);
            if (g.kind == 2) {
                for (size_t i = 0; i < D; ++i) {
                    int a = (i >> (n - 1 - g.q)) & 1, b = (i >> (n - 2 - g.q)) & 1;
                    double sgn = (a & b) ? -1 : 1;
                    for (size_t j = 0; j < D; ++j) Nt[i * D + j] = sgn * Mt[i * D + j];
                }
            } else {
                const M2 &G = raw[w][g.kind == 3 ? 0 : g.raw];
                int sh = n - 1 - g.q;
                for (size_t i = 0; i < D; ++i) {
                    int bi = (i >> sh) & 1;
                    for (int bo = 0; bo < 2; ++bo) {
                        size_t i2 = (i & ~((size_t)1 << sh)) | ((size_t)bo << sh);
                        for (size_t j = 0; j < D; ++j) Nt[i2 * D + j] += G.m[2 * bo + bi] * Mt[i * D + j];
                    }
                }
            }
            Mt.swap(Nt);
        }
        return Mt;
    };
    auto Ud = build(0), Vd = build(1);
    cd tr = 0; for (size_t k = 0; k < D * D; ++k) tr += std::conj(Ud[k]) * Vd[k];
    printf("n=%d L=%d bits=%d maps=%zu: spiral %.12f%+.12fi dense %.12f%+.12fi  |diff| %.2e\n", n, L, B, P.maps.size(),
           tr_sp.real(), tr_sp.imag(), tr.real(), tr.imag(), std::abs(tr_sp - tr));
    return std::abs(tr_sp - tr) <= 1e-12 * std::max(1.0, std::abs(tr)) ? 0 : 1;
}
