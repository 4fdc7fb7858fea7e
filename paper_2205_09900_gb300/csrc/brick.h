// brick.h -- brickwork fast path: closed-form dual-circuit sweep.
//
// For a brickwork pair of depth l >= 2, U^dagger V after the middle and cyclic
// merges is a cyclic brickwork of 2m = 2(l-1) layers; position tau holds the
// layer acting on bonds of parity (tau+1) mod 2:
//   tau = 0..l-3       V's layer tau+2
//   tau = l-2          U_l^dagger V_l          (middle merge)
//   tau = l-1..2l-4    U's layer 2l-2-tau, daggered
//   tau = 2l-3         V_1 U_1^dagger          (cyclic merge)
// Every interior qubit meets one gate per position, so its wire has 2m
// segments (segment tau precedes position tau).  The boundary at a bond is a
// state over the 2m segment bits of one qubit, bit tau = segment tau, and
// sweeping across bond b applies each bond-b gate G at position tau as an
// in-place 4x4 map on bits (tau, tau+1 mod 2m):
//   left sweep  M[(x_tau x_tau+1),(y_tau y_tau+1)]  = G[(y_tau+1 x_tau+1),(y_tau x_tau)]
//   right sweep M'[(y_tau y_tau+1),(x_tau x_tau+1)] = G[(y_tau+1 x_tau+1),(y_tau x_tau)]
// (y: qubit b, x: qubit b+1; 2-bit index e = w_tau + 2 w_tau+1).  The chain
// ends start from the product state prod delta(w_tau, w_tau+1) over the
// positions where the end qubit is idle.  The left sweep covers bonds
// 0..cut-1, the right sweep bonds n-2..cut; both end on qubit cut's segments
// and meet in a plain dot product.  The bit order is the ring order of the
// segments, so a contiguous cyclic arc of bits is a light-cone tile.
#pragma once
#include <cstdint>
#include <vector>

#include "fp_internal.h"

namespace fpk {

struct BrickGate {      // one gate inside a tile pass
    uint8_t layer;      // layer index within the side
    uint8_t j;          // gate index within the layer (tau = 2j + parity)
    uint8_t a, b;       // tile-local bits of segments tau and tau+1
};

struct BrickPass {
    int32_t gate_off, n_gates;
    uint32_t smask;     // physical bits held by the tile
    int32_t rp_off, n_rp;   // register passes (RegPass) of this tile pass
    int32_t rg_off;         // first RegGate of this tile pass
    // shared-memory layout of the tile: element i sits at i ^ s(i >> 4), s
    // linear over GF(2) into the low 4 bits, s of tile bit 4 + j = swz[j];
    // chosen per pass so that the 16 lanes of a half-warp reading one
    // register window hit 16 distinct 8-byte bank pairs
    uint8_t swz[12];
};

// One register pass inside a tile pass: every thread holds 2^r amplitudes
// spanning the window bits (r ring-consecutive tile bits) and applies the
// window gates in registers.  Gate g of the window acts on window bits
// (type, type+1); `slot` indexes the tile pass's gate list (its map).
constexpr int kMaxWin = 5;
struct RegPass {
    uint8_t win[kMaxWin];     // tile-local bits in ring order
    uint8_t srt[kMaxWin];     // the same bits ascending
    uint8_t r;
    uint8_t n_gates;
    int16_t gate_off;         // into the RegGate pool
};
struct RegGate {
    uint8_t type;
    uint8_t slot;
};

struct BrickDev {       // uniform over a sub-batch (one depth)
    int32_t n, l, m, N, cut;
    int32_t kind;             // 0: brickwork (l = depth), 1: HEA (l = L)
    int32_t n_layers[2];      // brickwork: side 0 bonds 0..cut-1, side 1 bonds n-2..cut;
                              // HEA: two layers per qubit (see below)
    int32_t delta_par[2];     // brickwork: delta(w_tau, w_tau+1) for tau of this parity at
                              // the chain end; HEA: the chain ends start from all ones
    int32_t pass_off[2], n_passes[2];
    int32_t tile_bits;        // K of the tiled path (0: whole state in one CTA)
};

// Tensor-core form of a register window (tile passes of kTcTile bits,
// windows of kMaxWin bits): the window's gates fused into one dense 32 x 32
// complex matrix W, applied to the tile viewed as a [128 rows x 32] complex
// matrix (rows: the other tile bits) by tcgen05 MMAs.  cb[b] is the byte
// offset contributed by tile-local bit b to an element's address in the MMA
// operand layout of this window (K-major, 128-byte swizzle; the layout is
// linear over GF(2), so an address is the XOR of its bits' contributions).
constexpr int kTcTile = 12;
constexpr int kTcRows = kTcTile - kMaxWin;
struct TcWin {
    uint8_t win[kMaxWin];     // tile-local bit of window position k (ring order)
    uint8_t row[kTcRows];     // tile-local bits of the row index, ascending
    uint32_t cb[kTcTile];
    // store order of the scatter from this window's result into the next
    // window's operand: lane L (bits 0-3) visits its outputs u ^ rot(L),
    // rot bit i = parity(L & (rotm >> 4i)), chosen on the host so that the 16
    // lanes of a half-warp hit 16 distinct 8-byte bank pairs (or as few
    // repeats as the layouts allow)
    uint16_t rotm;
    // tensor-memory operand form (brick_tcm_pass_kernel): the byte offset of
    // tile-local bit b in the 32 KB shared-memory exchange buffer through which
    // this window's input arrives (window 0: the tile loaded from the boundary,
    // lanes storing consecutive tile indices; window k: window k-1's results).
    // The addresses are linear over GF(2); bits 3-6 (the 8-byte bank pair) give
    // the storing lanes' 4 bits and this window's row positions 0-3 (the
    // loading lanes) 16 distinct bank pairs each, the 8 tile bits outside the
    // storing lanes' 4 fill bits 7-14 in ascending order.
    uint32_t xcb[kTcTile];
};
// The exchange addresses of one window for the tensor-memory operand form, by
// thread position: a drain thread (warp w of 8, lane l) holds row 32 (w mod 4)
// + l and window indices 16 (w / 4) + u, u = 0..15; its address of element u
// is lane[l] ^ warp[w] ^ (the c[k] of the set bits k of u).  ld: this window's
// operand, loaded through its own map xcb; st: this window's result, stored
// through the next window's map (zero for a pass's last window).
struct TcXa {
    uint32_t ld_lane[32], st_lane[32];
    uint32_t ld_warp[8], st_warp[8];
    uint32_t ld_c[4], st_c[4];
};
// A-operand byte address of element (row r, window index j): complex j
// occupies K columns 2j (re), 2j+1 (im); K splits into two 128-byte regions of
// 128 rows; 16-byte chunk c of row r sits at chunk c ^ (r % 8).
FP_HD uint32_t tc_addr(uint32_t r, uint32_t j) {
    return (j >> 4) * 16384u + r * 128u + ((((j >> 1) & 7u) ^ (r & 7u)) << 4) + (j & 1u) * 8u;
}
// Device copies of a plan's schedule (gates and register passes).
struct BrickDevPlan {
    const BrickGate *gates;
    const RegPass *rpasses;
    const RegGate *rgates;
    const TcWin *tcwins;    // persist >= 2: one per register pass
    const TcXa *tcxa;       // persist == 4: one per register pass
    int *err_flag;          // persist >= 2: raised by a kernel whose bounded wait ran out
    int win_bits;
    int threads;
    int persist;        // 1: persistent double-buffered tile passes; 3, 4: tensor-core windows (fp_brick_variant)
};

struct BrickHostPlan {
    BrickDev dev;
    std::vector<BrickPass> passes;   // side 0 passes, then side 1 passes
    std::vector<BrickGate> gates;
    std::vector<RegPass> rpasses;
    std::vector<RegGate> rgates;
};

// Brickwork: the bond that layer t of a side sweeps.
FP_HD int brick_bond(const BrickDev &d, int side, int t) { return side == 0 ? t : d.n - 2 - t; }
// Pairing of layer t: gates on bits (2j + p, 2j + p + 1 mod N).
FP_HD int layer_parity(const BrickDev &d, int side, int t) {
    return d.kind == 0 ? (brick_bond(d, side, t) + 1) % 2 : t % 2;
}
// Maps of a pair are stored [side][layer][j]: index of gate j of layer t.
FP_HD int map_index(const BrickDev &d, int side, int t, int j) {
    return ((side ? d.n_layers[0] : 0) + t) * d.m + j;
}
FP_HD int maps_per_pair(const BrickDev &d) { return (d.n_layers[0] + d.n_layers[1]) * d.m; }
// HEA (kind 1).  U^dagger V after the merges is a cycle of 2L-2 rotation
// slots per qubit with a CZ ladder after each: slot s = 0: R_1^V R_1^U^dagger,
// s = 1..L-2: R_{s+1}^V, s = L-1: R_L^U^dagger R_L^V, s = L..2L-3:
// R_{2L-1-s}^U^dagger.  Segment s of a wire runs from slot s through ladder s
// to slot s+1, so the boundary is a state over the 2L-2 segments of one qubit.
// Sweeping qubit q multiplies by its rotations, R_{q,s}[y_s, y_{s-1}] (a
// diagonal map on bits (s-1, s)), then crosses the CZ ladder, an
// unnormalised Hadamard [[1,1],[1,-1]] on every bit.  As brickwork layers:
// layer 2i: diagonal maps on pairs (2j, 2j+1) (slots 2j+1); layer 2i+1: the
// diagonal maps on pairs (2j+1, 2j+2) (slots 2j+2) followed by H x H.  Side 0
// sweeps qubits 0..cut-1; side 1 qubits n-1..cut+1 and finally qubit cut's
// rotations without a ladder.

BrickHostPlan make_brick_plan(int n, int l, int tile_bits, int low_bits, int win_bits, int kind = 0);
// Tensor-core window tables (one per register pass) of a plan with kTcTile-bit
// tiles and kMaxWin-bit windows.
std::vector<TcWin> make_tc_windows(const BrickHostPlan &P);
// Per-thread exchange address tables of those windows (one per register pass).
std::vector<TcXa> make_tc_xaddr(const BrickHostPlan &P, const std::vector<TcWin> &W);

}  // namespace fpk
