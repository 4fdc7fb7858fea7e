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
    int32_t n_layers[2];      // side 0: bonds 0..cut-1; side 1: bonds n-2..cut
    int32_t delta_par[2];     // delta(w_tau, w_tau+1) for tau of this parity at the chain end
    int32_t pass_off[2], n_passes[2];
    int32_t tile_bits;        // K of the tiled path (0: whole state in one CTA)
};

// Device copies of a plan's schedule (gates and register passes).
struct BrickDevPlan {
    const BrickGate *gates;
    const RegPass *rpasses;
    const RegGate *rgates;
    int win_bits;
    int threads;
};

struct BrickHostPlan {
    BrickDev dev;
    std::vector<BrickPass> passes;   // side 0 passes, then side 1 passes
    std::vector<BrickGate> gates;
    std::vector<RegPass> rpasses;
    std::vector<RegGate> rgates;
};

// Layer parity of layer t of a side, and the bond it sweeps.
FP_HD int brick_bond(const BrickDev &d, int side, int t) { return side == 0 ? t : d.n - 2 - t; }

BrickHostPlan make_brick_plan(int n, int l, int tile_bits, int low_bits, int win_bits);

}  // namespace fpk
