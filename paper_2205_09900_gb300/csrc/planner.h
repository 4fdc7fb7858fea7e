// planner.h -- host planner: from the gate layout of a circuit pair to the two
// boundary-sweep programs that contract the closed trace network of U^dagger V.
#pragma once
#include <string>
#include <vector>

#include "fp_internal.h"

namespace fpk {

// One gate of a circuit as laid out by an ensemble (values come from the sampler).
struct GateSlot {
    int kind;   // 0: 2-qubit on bond q (raw gate), 1: 1-qubit on q (raw gate),
                // 2: constant diagonal 2-qubit (CZ) on bond q, 3: 1-qubit on q
                // (raw gate) that is the same constant involution in U and V
                // (the Hadamard of a CNOT): two of them meeting cancel
    int q;
    int raw;    // raw gate index within the circuit, -1 for constants
};

struct HostPlan {
    int n = 0;
    int n_raw = 0;
    int raw_kind = RAW_HAAR4;
    std::vector<MergeRef> refs;
    std::vector<MergeItem> merges;
    std::vector<DevOp> ops;          // left sweep, then right sweep
    std::vector<DevRecipe> recipes;  // one per op
    int n_left = 0, n_right = 0;
    int bits_max = 0, bits_final = 0, left_final_buf = 0;
    std::vector<uint8_t> dot_perm;
    double prefactor = 1.0;
    double cost = 0.0;               // complex multiply-adds per pair
    // brickwork fast-path description (valid when brick_ok)
    bool brick_ok = false;
    int brick_m = 0;                 // gates per bond = bits/2
    std::string error;               // non-empty: planning failed
    bool infeasible = false;
};

std::vector<GateSlot> layout_brickwork(int n, int l);
std::vector<GateSlot> layout_hea(int n, int L);
std::vector<GateSlot> layout_local(int n, const std::vector<int> &bonds);
// The paper's HEA (Fig. 2c): RY(pi/4) wall, then per layer Pauli rotations and
// CNOT walls on the even, then the odd bonds (CZ walls when `cz`).  A CNOT is
// laid out as H(target) CZ H(target) (H of kind 3), so that its control wire
// stays uncut.
std::vector<GateSlot> layout_hea_pauli(int n, int L, bool cz);

// Spiral program (the paper's HEA with CNOT walls, and any circuit of 1-qubit
// gates and CZs whose wires alternate between taps on the left and the right
// bond).  The state holds one variable per CZ of a bond (M bits) plus an
// auxiliary bit M; a qubit's wire, a ring of segments each tapped by one CZ, is
// absorbed by M+1 in-place 4x4 maps (planner.cpp explains the recipes).
struct SpiralPlan {
    bool ok = false;
    int bits = 0;               // M + 1
    int first_bit = 0;          // start state delta(aux, bit first_bit)
    std::vector<MergeRef> refs;
    std::vector<MergeItem> merges;
    std::vector<SpiralMap> maps;
    std::string why;            // why not, when !ok
};
SpiralPlan make_spiral_plan(int n, const std::vector<GateSlot> &U, const std::vector<GateSlot> &V, int raw_kind);
// Consecutive maps grouped into windows of R state bits (R <= kSpiralMaxWin,
// padded with the lowest other bits); ij[k]: map k's window-local (low, high)
// bits.  `split` (0, 1, 2) cluster bits are the state bits fewest windows touch
// (returned ascending in h[0], h[1]; -1 when unused); every window gets its
// addressing (SpiralWin).  Needs bits - R - split >= 4.
void spiral_windows(const SpiralPlan &P, int R, int split, std::vector<SpiralWin> &wins, std::vector<uint8_t> &ij,
                    int h[2]);

// Plan the contraction of Tr(U^dagger V).  `cut`: the left sweep owns bonds
// 0..cut-1 and the 1-qubit gates of qubits 0..cut-1, the right sweep the rest.
HostPlan make_plan(int n, const std::vector<GateSlot> &U, const std::vector<GateSlot> &V,
                   int raw_kind, int n_raw, int cut, int max_bits);

}  // namespace fpk
