// tc_pass_check.cpp -- host emulation of the tensor-core tile pass of the
// brickwork sweep (kernels_brick_tc.cu), independent of the GPU.
//
// For a brickwork plan with 12-bit tiles and 5-bit windows (brick_plan.cpp:
// make_brick_plan, make_tc_windows) and random 4x4 maps, one side's boundary
// is swept twice in FP64:
//   reference  every window's gates applied one by one on the full state;
//   emulation  the kernel's data movement: tiles gathered into the A operand
//              through the window-0 address tables, per window the dense
//              32 x 32 matrix W built column by column and stored in the B
//              operand layout, the MMA read through the hardware's view of
//              the K-major 128-byte-swizzled operands (row r, K column k at
//              region k/32, row offset 128 r, 16-byte chunk (k/4 mod 8) ^ (r mod 8)),
//              D = A B^T, then every thread's 16 results (8 warps) scattered through the
//              XOR address tables into the next window's operand or the boundary.
// Every operand address is checked to be in bounds and every window layout
// to be a bijection.  Exit status 1 if the two sweeps differ by more than
// 1e-12 (relative to the largest amplitude) or an address check fails.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <vector>

#include "brick.h"

using namespace fpk;
typedef std::complex<double> cd;

static int fails = 0;
#define CHECK(c, ...)                 \
    do {                              \
        if (!(c)) {                   \
            printf(__VA_ARGS__);      \
            printf("\n");             \
            ++fails;                  \
        }                             \
    } while (0)

static uint32_t hw_a(uint32_t r, uint32_t k) {   // A operand: 128 rows, K regions of 16 KB
    return (k >> 5) * 16384u + r * 128u + ((((k >> 2) & 7u) ^ (r & 7u)) << 4) + (k & 3u) * 4u;
}
static uint32_t hw_b(uint32_t n, uint32_t k) {   // B operand: 64 rows, K regions of 8 KB
    return (k >> 5) * 8192u + n * 128u + ((((k >> 2) & 7u) ^ (n & 7u)) << 4) + (k & 3u) * 4u;
}

static void apply4(std::vector<cd> &s, int N, int pa, int pb, const cd *T) {
    const uint32_t S = 1u << N;
    for (uint32_t i = 0; i < S; ++i) {
        if ((i >> pa) & 1u || (i >> pb) & 1u) continue;
        const uint32_t ia = 1u << pa, ib = 1u << pb;
        cd x[4] = {s[i], s[i | ia], s[i | ib], s[i | ia | ib]};
        cd y[4];
        for (int o = 0; o < 4; ++o) y[o] = T[4 * o] * x[0] + T[4 * o + 1] * x[1] + T[4 * o + 2] * x[2] + T[4 * o + 3] * x[3];
        s[i] = y[0]; s[i | ia] = y[1]; s[i | ib] = y[2]; s[i | ia | ib] = y[3];
    }
}

// 8-byte bank pair (address bits 3-6) of each of 16 lanes' addresses: all distinct?
static bool distinct_banks(const uint32_t *a) {
    unsigned seen = 0;
    for (int i = 0; i < 16; ++i) seen |= 1u << ((a[i] >> 3) & 15u);
    return seen == 0xFFFFu;
}

int main(int argc, char **argv) {
    const int n = atoi(argv[1]), l = atoi(argv[2]);
    // "tcm": the tensor-memory operand form (brick_tcm_pass_kernel): every window's input
    // through the shared-memory exchange buffer (TcWin::xcb) into a [128 x 32] complex
    // operand held by 8 warps x 32 lanes x 16 window indices, results stored back by
    // the same threads into the next window's exchange buffer; every address also
    // recomputed from the per-thread tables (TcXa) the kernel reads
    const bool tcm = argc > 3 && std::string(argv[3]) == "tcm";
    BrickHostPlan P = make_brick_plan(n, l, kTcTile, 3, kMaxWin, 0);   // the plan the tensor-core pass runs
    const BrickDev &d = P.dev;
    const int N = d.N;
    const uint32_t S = 1u << N;
    CHECK(d.tile_bits == kTcTile && N >= kTcTile + 1, "plan is not tiled with %d-bit tiles", kTcTile);
    std::vector<TcWin> W = make_tc_windows(P);
    std::vector<TcXa> XA = make_tc_xaddr(P, W);   // the tensor-memory kernel's per-thread tables
    std::mt19937_64 rng(1000 * n + l);
    std::normal_distribution<double> N01;
    // random unitary maps (Gram-Schmidt on complex Gaussian columns): norms stay 1 over the sweep
    std::vector<cd> maps((size_t)maps_per_pair(d) * 16);
    for (size_t g = 0; g < maps.size() / 16; ++g) {
        cd *M = &maps[g * 16];
        for (int c = 0; c < 4; ++c) {
            cd col[4];
            for (int r = 0; r < 4; ++r) col[r] = cd(N01(rng), N01(rng));
            for (int c2 = 0; c2 < c; ++c2) {
                cd dot = 0;
                for (int r = 0; r < 4; ++r) dot += std::conj(M[4 * r + c2]) * col[r];
                for (int r = 0; r < 4; ++r) col[r] -= dot * M[4 * r + c2];
            }
            double nn = 0;
            for (int r = 0; r < 4; ++r) nn += std::norm(col[r]);
            for (int r = 0; r < 4; ++r) M[4 * r + c] = col[r] / std::sqrt(nn);
        }
    }
    int max_rp = 0;
    for (int side = 0; side < 2; ++side) {
        std::vector<cd> ref(S), emu(S);
        for (uint32_t i = 0; i < S; ++i) ref[i] = emu[i] = cd(N01(rng), N01(rng));
        for (int p = 0; p < d.n_passes[side]; ++p) {
            const BrickPass &ps = P.passes[d.pass_off[side] + p];
            max_rp = std::max(max_rp, ps.n_rp);
            int pos[32], k = 0;
            for (int b = 0; b < N; ++b)
                if (ps.smask & (1u << b)) pos[k++] = b;
            CHECK(k == kTcTile, "pass %d holds %d bits", p, k);
            auto mapp = [&](int slot) {
                const BrickGate &g = P.gates[ps.gate_off + slot];
                return &maps[(size_t)map_index(d, side, g.layer, g.j) * 16];
            };
            // reference: window by window, gate by gate, on the whole state
            for (int w = 0; w < ps.n_rp; ++w) {
                const RegPass &rp = P.rpasses[ps.rp_off + w];
                CHECK(rp.r == kMaxWin, "window of %d bits", rp.r);
                for (int g = 0; g < rp.n_gates; ++g) {
                    const RegGate &rg = P.rgates[rp.gate_off + g];
                    apply4(ref, N, pos[rp.win[rg.type]], pos[rp.win[rg.type + 1]], mapp(rg.slot));
                }
            }
            // window layouts are bijections onto the 4096 8-byte slots of a 32 KB operand
            for (int w = 0; w < ps.n_rp; ++w) {
                const TcWin &tw = W[ps.rp_off + w];
                std::vector<char> hit(4096, 0);
                for (uint32_t i = 0; i < 4096; ++i) {
                    uint32_t a = 0;
                    for (int b = 0; b < kTcTile; ++b)
                        if ((i >> b) & 1u) a ^= tw.cb[b];
                    CHECK(a < 32768 && a % 8 == 0, "address %u out of the operand", a);
                    if (a < 32768) hit[a / 8]++;
                }
                CHECK(std::count(hit.begin(), hit.end(), 1) == 4096, "window %d layout is not a bijection", w);
            }
            // the window matrices, as tc_wmat_kernel builds and stores them
            std::vector<std::vector<double>> B(ps.n_rp, std::vector<double>(8192 / 1, 0.0));
            for (int w = 0; w < ps.n_rp; ++w) {
                const RegPass &rp = P.rpasses[ps.rp_off + w];
                std::vector<char> seen(4096, 0);
                for (int j = 0; j < 32; ++j) {
                    std::vector<cd> v(32, 0.0);
                    v[j] = 1.0;
                    for (int g = 0; g < rp.n_gates; ++g) {
                        const RegGate &rg = P.rgates[rp.gate_off + g];
                        apply4(v, 5, rg.type, rg.type + 1, mapp(rg.slot));
                    }
                    for (int o = 0; o < 32; ++o) {
                        const uint32_t a0 = hw_b(2 * o, 2 * j), a1 = hw_b(2 * o + 1, 2 * j);
                        CHECK(a0 < 16384 && a1 < 16384, "B address out of range");
                        // float pairs at a0: (re, -im); at a1: (im, re)
                        B[w][a0 / 4] = v[o].real(); B[w][a0 / 4 + 1] = -v[o].imag();
                        B[w][a1 / 4] = v[o].imag(); B[w][a1 / 4 + 1] = v[o].real();
                        seen[a0 / 4]++; seen[a0 / 4 + 1]++; seen[a1 / 4]++; seen[a1 / 4 + 1]++;
                    }
                }
                CHECK(std::count(seen.begin(), seen.end(), 1) == 4096, "B layout is not a bijection");
            }
            uint32_t gcb[kTcTile];
            for (int b = 0; b < kTcTile; ++b) gcb[b] = 1u << pos[b];
            if (tcm) {
                const uint32_t ntiles = 1u << (N - kTcTile);
                auto xaddr = [](const uint32_t *cb, const uint8_t *rows, uint32_t r, const uint8_t *win, uint32_t j) {
                    uint32_t a = 0;
                    for (int q = 0; q < kTcRows; ++q)
                        if ((r >> q) & 1u) a ^= cb[rows[q]];
                    for (int q = 0; q < kMaxWin; ++q)
                        if ((j >> q) & 1u) a ^= cb[win[q]];
                    return a;
                };
                for (uint32_t t = 0; t < ntiles; ++t) {
                    uint32_t base = 0, tt = t;
                    for (int b = 0; b < N; ++b)
                        if (!(ps.smask & (1u << b))) { base |= (tt & 1u) << b; tt >>= 1; }
                    std::vector<cd> X(4096), X2(4096);
                    const TcWin &w0 = W[ps.rp_off];
                    for (uint32_t i0 = 0; i0 < 4096; i0 += 16) {   // the tile load, 16 lanes at a time
                        uint32_t ad[16];
                        for (uint32_t q = 0; q < 16; ++q) {
                            const uint32_t i = i0 + q;
                            uint32_t phys = base, a = 0;
                            for (int b = 0; b < kTcTile; ++b)
                                if ((i >> b) & 1u) { phys |= 1u << pos[b]; a ^= w0.xcb[b]; }
                            CHECK(a < 32768 && a % 8 == 0, "exchange address %u", a);
                            X[(a / 8) & 4095] = emu[phys];
                            ad[q] = a;
                        }
                        CHECK(distinct_banks(ad), "tile load: repeated bank pair");
                    }
                    for (int w = 0; w < ps.n_rp; ++w) {
                        const TcWin &cw = W[ps.rp_off + w];
                        // operand rows: warp (0..7) and lane give the row, u the window index
                        std::vector<double> Ar(128 * 64);
                        for (int warp = 0; warp < 8; ++warp)
                            for (int u = 0; u < 16; ++u)
                                for (int h = 0; h < 2; ++h) {
                                    uint32_t ad[16];
                                    for (int q = 0; q < 16; ++q) {
                                        const uint32_t r = 32u * (warp & 3) + 16u * h + q, j = 16u * (warp >> 2) + u;
                                        ad[q] = xaddr(cw.xcb, cw.row, r, cw.win, j);
                                        const TcXa &xa = XA[ps.rp_off + w];
                                        uint32_t tab = xa.ld_lane[16 * h + q] ^ xa.ld_warp[warp];
                                        for (int k = 0; k < 4; ++k)
                                            if ((u >> k) & 1) tab ^= xa.ld_c[k];
                                        CHECK(tab == ad[q], "window %d: load table differs from the map", w);
                                        const cd x = X[(ad[q] / 8) & 4095];
                                        Ar[r * 64 + 2 * j] = x.real();
                                        Ar[r * 64 + 2 * j + 1] = x.imag();
                                    }
                                    CHECK(distinct_banks(ad), "window %d load: repeated bank pair", w);
                                }
                        std::vector<double> D(128 * 64);
                        for (uint32_t r = 0; r < 128; ++r)
                            for (uint32_t nn = 0; nn < 64; ++nn) {
                                double acc = 0;
                                for (uint32_t kk = 0; kk < 64; ++kk) acc += Ar[r * 64 + kk] * B[w][hw_b(nn, kk) / 4];
                                D[r * 64 + nn] = acc;
                            }
                        const bool last = w + 1 == ps.n_rp;
                        std::vector<char> hit(4096, 0);
                        for (int warp = 0; warp < 8; ++warp)
                            for (int u = 0; u < 16; ++u)
                                for (int h = 0; h < 2; ++h) {
                                    uint32_t ad[16];
                                    for (int q = 0; q < 16; ++q) {
                                        const uint32_t r = 32u * (warp & 3) + 16u * h + q, o = 16u * (warp >> 2) + u;
                                        const cd y(D[r * 64 + 2 * o], D[r * 64 + 2 * o + 1]);
                                        if (last) {   // straight to the boundary
                                            const uint32_t g = xaddr(gcb, cw.row, r, cw.win, o);
                                            CHECK((g & base) == 0 && g < S, "boundary index out of the tile");
                                            emu[base | g] = y;
                                            ad[q] = 8u * q;
                                        } else {
                                            const TcWin &nx = W[ps.rp_off + w + 1];
                                            ad[q] = xaddr(nx.xcb, cw.row, r, cw.win, o);
                                            const TcXa &xa = XA[ps.rp_off + w];
                                            uint32_t tab = xa.st_lane[16 * h + q] ^ xa.st_warp[warp];
                                            for (int k = 0; k < 4; ++k)
                                                if ((u >> k) & 1) tab ^= xa.st_c[k];
                                            CHECK(tab == ad[q], "window %d: store table differs from the map", w);
                                            CHECK(ad[q] < 32768 && ad[q] % 8 == 0, "exchange address %u", ad[q]);
                                            X2[(ad[q] / 8) & 4095] = y;
                                            hit[(ad[q] / 8) & 4095]++;
                                        }
                                    }
                                    CHECK(distinct_banks(ad), "window %d store: repeated bank pair", w);
                                }
                        if (!last) {
                            CHECK(std::count(hit.begin(), hit.end(), 1) == 4096, "exchange %d is not a bijection", w);
                            X.swap(X2);
                        }
                    }
                }
                continue;
            }
            // emulation of every tile (one per CTA)
            const uint32_t ntiles = 1u << (N - kTcTile);
            for (uint32_t t = 0; t < ntiles; ++t) {
                uint32_t base = 0, tt = t;
                for (int b = 0; b < N; ++b)
                    if (!(ps.smask & (1u << b))) { base |= (tt & 1u) << b; tt >>= 1; }
                std::vector<double> A(8192, 0.0);   // one 32 KB operand as floats
                const TcWin &w0 = W[ps.rp_off];
                for (uint32_t i = 0; i < 4096; ++i) {
                    uint32_t phys = base, a = 0;
                    for (int b = 0; b < kTcTile; ++b)
                        if ((i >> b) & 1u) { phys |= 1u << pos[b]; a ^= w0.cb[b]; }
                    A[a / 4] = emu[phys].real();
                    A[a / 4 + 1] = emu[phys].imag();
                }
                for (int w = 0; w < ps.n_rp; ++w) {
                    // MMA: D[r][n] = sum_k A(r, k) B(n, k) through the hardware's operand view
                    std::vector<double> D(128 * 64);
                    for (uint32_t r = 0; r < 128; ++r)
                        for (uint32_t nn = 0; nn < 64; ++nn) {
                            double acc = 0;
                            for (uint32_t kk = 0; kk < 64; ++kk) acc += A[hw_a(r, kk) / 4] * B[w][hw_b(nn, kk) / 4];
                            D[r * 64 + nn] = acc;
                        }
                    const TcWin &cw = W[ps.rp_off + w];
                    const bool last = w + 1 == ps.n_rp;
                    const uint32_t *cbn = last ? gcb : W[ps.rp_off + w + 1].cb;
                    std::vector<double> A2(8192, 0.0);
                    for (int warp = 0; warp < 8; ++warp)
                        for (int lane = 0; lane < 32; ++lane) {
                            const uint32_t r = 32u * (warp & 3) + lane;
                            uint32_t bs = 0;
                            for (int q = 0; q < kTcRows; ++q)
                                if ((r >> q) & 1u) bs ^= cbn[cw.row[q]];
                            const int half = warp >> 2;
                            if (half) bs ^= cbn[cw.win[4]];
                            // the kernel visits output u ^ rot at step u (rot by lane, TcWin::rotm)
                            const uint32_t rm = last ? 0u : cw.rotm, l4 = (uint32_t)lane & 15u;
                            int rot = 0;
                            for (int i = 0; i < 3; ++i)
                                rot |= (__builtin_popcount(l4 & ((rm >> (4 * i)) & 15u)) & 1) << i;
                            for (int step = 0; step < 16; ++step) {
                                const int u = step ^ rot;
                                uint32_t a = bs;
                                for (int q = 0; q < 3; ++q)
                                    if ((rot >> q) & 1) a ^= cbn[cw.win[q]];
                                for (int q = 0; q < 4; ++q)
                                    if ((step >> q) & 1) a ^= cbn[cw.win[q]];
                                const uint32_t col = 32u * half + 2u * u;
                                const double x = D[r * 64 + col], y = D[r * 64 + col + 1];
                                if (last) {
                                    CHECK((a & ~(S - 1)) == 0 && (a & base) == 0, "boundary index out of the tile");
                                    emu[base | a] = cd(x, y);
                                } else {
                                    CHECK(a < 32768 && a % 8 == 0, "operand address %u", a);
                                    A2[a / 4] = x;
                                    A2[a / 4 + 1] = y;
                                }
                            }
                        }
                    if (!last) A.swap(A2);
                }
            }
        }
        double mx = 0, dmax = 0;
        for (uint32_t i = 0; i < S; ++i) {
            mx = std::max(mx, std::abs(ref[i]));
            dmax = std::max(dmax, std::abs(ref[i] - emu[i]));
        }
        printf("n=%d l=%d side %d: %d passes, max |ref| %.3e, max diff %.3e\n", n, l, side, d.n_passes[side], mx, dmax);
        CHECK(dmax <= 1e-12 * mx, "side %d: emulation differs from the gate-by-gate sweep", side);
    }
    printf("max windows per pass %d\n", max_rp);
    return fails ? 1 : 0;
}
