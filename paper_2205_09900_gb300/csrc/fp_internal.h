// fp_internal.h -- structures shared by the host planner and the sm_103a kernels.
#pragma once
#include <cstdint>
#include <cstddef>

#include "fp.h"

#if defined(__CUDACC__)
#define FP_HD __host__ __device__ __forceinline__
#else
#define FP_HD inline
#endif

namespace fpk {

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), used on host (per-pair
// depth, local-circuit bonds) and device (gate sampling).  Keying is stated
// in fp.h.
// ---------------------------------------------------------------------------
struct U64x4 { uint64_t x[4]; };

FP_HD void mul_hilo(uint64_t a, uint64_t b, uint64_t &hi, uint64_t &lo) {
#if defined(__CUDA_ARCH__)
    lo = a * b;
    hi = __umul64hi(a, b);
#else
    unsigned __int128 p = (unsigned __int128)a * b;
    hi = (uint64_t)(p >> 64);
    lo = (uint64_t)p;
#endif
}

FP_HD U64x4 philox(uint64_t seed, uint64_t c0, uint64_t c1, uint64_t pair, uint64_t stream) {
    uint64_t c[4] = {c0, c1, pair, stream};
    uint64_t k0 = seed, k1 = 0;
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0, lo0, hi1, lo1;
        mul_hilo(0xD2E7470EE14C6C93ULL, c[0], hi0, lo0);
        mul_hilo(0xCA5A826395121157ULL, c[2], hi1, lo1);
        uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += 0x9E3779B97F4A7C15ULL;
        k1 += 0xBB67AE8584CAA73BULL;
    }
    U64x4 o;
    o.x[0] = c[0]; o.x[1] = c[1]; o.x[2] = c[2]; o.x[3] = c[3];
    return o;
}

FP_HD uint32_t pick(uint64_t x, uint32_t choices) {   // uniform index in [0, choices)
    return (uint32_t)(((x >> 32) * (uint64_t)choices) >> 32);
}

// ---------------------------------------------------------------------------
// Raw gates (as sampled) and merged gates live in 16-slot complex records:
// a 4x4 matrix row-major, or a 2x2 in slots 0..3.
// ---------------------------------------------------------------------------
// RAW_PAULI (the paper's HEA): raw 0 = Hadamard, raw 1..n = the RY(pi/4)
// wall, raw 1 + n + t n + q = rotation R_P(theta) of layer t on qubit q.
enum RawKind : int32_t { RAW_HAAR4 = 0, RAW_ROT2 = 1, RAW_DIAG4 = 2, RAW_PAULI = 3 };

// One raw-gate reference inside a merged product.
struct MergeRef {
    int32_t which;    // 0 = U, 1 = V
    int32_t gate;     // raw gate index within that circuit
    int32_t dagger;   // 1: use the conjugate transpose
    int32_t dim;      // 4 or 2
};

// A merged gate = product of refs[first .. first+count-1], refs[first] acting first.
struct MergeItem {
    int32_t first;
    int32_t count;
};

// One operation of a sweep program: multiply the state by a factor table over
// <= 4 binary variables, each consumed (summed, removed), kept, or new.
struct DevOp {
    uint8_t nc, nk, nn, b_in;
    uint8_t b_out, inplace2, pad0, pad1;
    uint8_t cons_pos[4];   // ascending positions in the input layout
    uint8_t keep_pos[4];   // positions in the output layout
    uint8_t new_pos[4];    // ascending positions in the output layout
};

// How to fill one op's table (16 entries, index e = cons | keep<<nc | new<<(nc+nk)).
struct DevRecipe {
    int32_t merged;        // merged gate id, or -1 for constants
    int32_t nent;          // 2^(nc+nk+nn)
    int8_t src[16][4];     // merged-gate slots summed into entry e (-1: unused)
    int8_t sgn[16][4];     // +1 / -1 weight of each summed slot (a fused CZ sign)
    double cre[16];        // constant entries (merged == -1)
    double cim[16];
};

// One 4x4 map of the spiral sweep (planner.cpp: make_spiral_plan).
enum SpiralType : uint8_t {
    SP_DIAG_BA = 0,   // delta(o, i) G[i_b][i_a]
    SP_START = 1,     // delta(o_a, o_b) H[o_b][i_b]                    (a = aux: copy, old aux summed)
    SP_MID = 2,       // F[o_a][i_a] G[o_b][o_a] H[o_b][i_b]
    SP_MID_AUX = 3,   // delta(o_b, i_b) F[o_a][i_a] G[o_b][o_a]
    SP_RL = 4,        // delta(o_a, i_a) G[o_b][i_a] H[o_b][i_b]
    SP_MID_RR = 5,    // F[o_a][i_a] G[o_b][o_a] delta(i_b, 0)
    SP_RR = 6,        // delta(o_a, i_a) G[o_b][i_a] delta(i_b, 0)
    SP_LL = 7,        // delta(o_a, 0) G[o_b][i_a] H[o_b][i_b]
    SP_LL_AUX = 8     // delta(o_a, 0) delta(o_b, i_b) G[i_b][i_a]
};
struct SpiralMap {
    uint8_t a, b;     // state bits of the map's low and high index bit
    uint8_t type;     // SpiralType
    uint8_t pad;
    int32_t f, g;     // merged 1-qubit items the recipe uses (-1: none)
};
// A register window of the spiral sweep: maps [first, first + n_maps) act only
// on the window's nb state bits (ascending); map k acts on window bits
// (ij[k] & 15, ij[k] >> 4) as its (low, high) index bits.
// The state is split over s = 0, 1 or 2 cluster bits h0 < h1: amplitude x
// lives in CTA rank (x_h0 + 2 x_h1) of a 2^s-CTA cluster at local index
// y = x without those bits, stored at the swizzled slot
// sw(y) = y ^ fold4(y >> 4) (fold4: XOR of the 4-bit chunks).  A CTA handles
// the window's groups t' = rank * G + t; the group base takes bit j of t' at
// state bit pos[j] (the four lane bits first, the cluster bits last, so that a
// window without cluster bits stays in its CTA).  Amplitude i of a group sits
// at slot sw(base) ^ (XOR of off[k] over the set bits k of i) in CTA
// rank(base) ^ (XOR of ctab[k]).
constexpr int kSpiralMaxWin = 5;
constexpr int kSpiralWinMaxMaps = 16;   // maps per window (staged in shared memory)
constexpr int kSpiralMaxPos = 24;
struct SpiralWin {
    uint8_t bits[kSpiralMaxWin];   // state bits of the window, ascending
    uint8_t nb;                    // window bits (the register block is 2^nb)
    uint8_t n_maps;
    uint8_t cross;                 // 1: the window holds a cluster bit
    uint8_t n_pos;                 // bits - nb
    uint8_t ctab[kSpiralMaxWin];   // rank contribution of each window bit (cluster bits)
    uint8_t pos[kSpiralMaxPos];
    uint16_t off[kSpiralMaxWin];   // sw(local unit vector) of each window bit (0: cluster bit)
    int32_t first;
};

// One pair of a batch.
struct PairInfo {
    uint64_t pair;        // global pair index (Philox counter word)
    int32_t plan;         // DevPlan index (generic path)
    int32_t n_raw;        // raw gates per circuit
    int64_t raw_off;      // first raw gate (16-slot records) of this pair
    int64_t merged_off;   // first merged gate (generic path)
    int64_t table_off;    // first op table (generic path)
    int64_t out;          // output slot in tr/kappa
};

// Device view of one plan (one topology).
struct DevPlan {
    int32_t n_left, n_right;       // ops in each sweep
    int32_t ops_off;               // first op in the op pool (left ops, then right ops)
    int32_t rec_off;               // first recipe in the recipe pool (same order)
    int32_t merge_off;             // first MergeItem in the merge pool
    int32_t n_merged;
    int32_t ref_off;               // MergeRef pool offset (MergeItem.first is relative)
    int32_t n_raw;                 // raw gates per circuit
    int32_t raw_kind;              // RawKind
    int32_t bits_max;              // largest state in either sweep
    int32_t bits_final;            // bits of the meeting boundary
    int32_t left_final_buf;        // 0/1: buffer holding the left result
    uint8_t dot_perm[FP_MAX_STATE_BITS];   // right-layout position of left bit k
    double prefactor;              // 2^(free wire loops)
    double cost;                   // estimated complex MACs per pair
    double sqrt_ops;               // sqrt(ops of the longer sweep), for the error estimate
};

}  // namespace fpk
