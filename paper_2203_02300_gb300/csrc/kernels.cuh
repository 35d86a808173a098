// Device-side types and constants of the AD-census matcher (arXiv 2203.02300, Sect. 4).
//
// Data layout in HBM (row-major, pixel index i = y*W + x):
//   rgbx[i]  uint32 r | g<<10 | b<<20          colour in three 10-bit fields (arm tests)
//   grey[i]  uint8  (77R + 150G + 29B + 128) >> 8
//   rec[y*rpitch + x]  uint4 {census bits 0-31, census bits 32-63,
//                    r | g<<8 | b<<16 | Lmin<<24, float bits of alpha(Lmin)*S}
//                    rows padded by kRPad records on both sides
//   arms[i]  uchar4 {left, right, up, down}
//   sh[i*dstride + j]  uint32 horizontal segment sum (fixed point) of
//                    disparity d0 + j (one pass of the d range)
//   best[i]  uint64 (aggregate << 32 | d), WTA state carried across passes
//
// Costs are carried in unsigned fixed point with scale S (an integer below
// 2^20, chosen so a full (2*L1+1)^2 region of costs <= 1 stays below 2^32).
// Prefix sums wrap modulo 2^32, and differences of prefix sums are exact
// region sums, so the Eq. 2 aggregation is exact integer arithmetic on the
// rounded per-pixel costs; only the Eq. 1 evaluation (FP32) and the rounding
// to fixed point differ from the real-valued definition.
#pragma once
#include <cuda.h>   // CUtensorMap (the encoder is reached through the runtime)
#include <cstdint>
#include <cuda_runtime.h>

namespace dco {

constexpr int kMaxL1 = 40;
constexpr int kTabAD = 768;   // entries of the AD table (sum of 3 abs diffs, 0..765)
constexpr int kTabCen = 96;   // entries of the census table (Hamming 0..64)
constexpr int kTabAlpha = 64; // alpha*S by Lmin, 0..kMaxL1
constexpr int kTabFloats = kTabAD + kTabCen + kTabAlpha;

// Record rows are padded by kRPad records on both sides, so a candidate
// x +- d with 0 <= d < 256 never leaves the allocation (its value is then
// discarded: the cost of a match outside the image is 1).
constexpr int kRPad = 256;

// Candidate planes (read by the cost pass's bulk copies): per image and
// row, the census words (uint2) and the colours (uint32) of the even
// columns, then of the odd columns, each half phw entries long (ceil(W / 2)
// rounded up to a multiple of 4, so every half starts on a 16-byte
// boundary); 16 bytes of slack after the last row.

// The cost H pass gives each warp kHSegCost columns of the prefix range (two
// half-warp segments of 16; one chunk per row up to kHMaxLen columns, else
// 512-column chunks), k_vcost each warp kHSegCost rows, the vote H pass
// segments of kHSeg; the V pass rows in segments of 1 << seglog.
constexpr int kHSegLog = 6, kHSeg = 1 << kHSegLog;
constexpr int kHSegCost = 32;
constexpr int kHNarrow = 20;     // warps of the cost H instantiation kept at two blocks per SM
constexpr int kHMaxLen = 1024;   // prefix columns one H block holds
constexpr int kVMaxLen = 1024;   // prefix rows one V block holds

struct PackArgs {
    const uint8_t *rgb[2];
    uint32_t *rgbx[2];
    uint8_t *grey[2];
    int npx, W;
    uint32_t k1;           // colour threshold tau1 in every 10-bit field (see kM9)
};

struct PrepArgs {
    const uint32_t *rgbx[2];
    const uint8_t *grey[2];
    uint4 *rec[2];         // first real record of row 0; row pitch rpitch
    uint2 *cen[2];         // candidate planes (census, colour): row y, column x at
    uint32_t *col[2];      //   y * 2 phw + (x & 1) * phw + (x >> 1)
    int phw;
    uchar4 *arms[2];
    const float *tables;   // alpha*S table at offset kTabAD + kTabCen
    int W, H, rpitch;
    int cw, ch;            // census window (odd)
    int L1, L2, tau1, tau2;
};

struct HArgs {
    const uint4 *rec[2];   // padded rows, pitch rpitch
    const uint2 *cen[2];   // candidate planes (PrepArgs)
    const uint32_t *col[2];
    int phw;
    int *status;           // device status word (a lost staging copy sets bit 0)
    int wait_limit;        // mbarrier polls before the staging copies are declared lost
    int skip_copy;         // failure test: arm the staging barrier but issue no copy
    const uchar4 *arms[2];
    uint32_t *sh[2];
    const float *tables;
    int W, H, D, rpitch;
    int d0, dc;            // this pass covers d in [d0, d0 + dc)
    int dstride;           // uint32 per pixel in sh (dc rounded up to 32)
    int ngroups;           // 32-disparity groups in the pass
    int L1;
    int chunk;             // output columns per block
    float S;               // fixed-point scale (integer valued)
    uint32_t Sint;
};

// horizontal pass of the parallax optimisation (Eq. 4): per-d vote counts
struct HVArgs {
    const int16_t *disp;   // map voted on, W x H, -1 = invalid
    const uchar4 *arms;    // reference-view arms {l, r, u, d}
    uint32_t *sh;          // count slices [y][x][dstride]
    int W, H, d0, dstride, L1, chunk;
};

// quarter-size input (Sect. 4): the two images of a pair, W x H -> W/2 x H/2
struct DownArgs {
    const uint8_t *src[2];
    uint8_t *dst[2];
    int W, H;
};

// sparse depth (Sect. 4.4) of a half-size map on the W x H grid
struct DepthArgs {
    const int16_t *disp;   // (H/2) x (W/2)
    float *out;            // W x H
    int W, H;
    float fb;              // f * B
};

// smoothing of the cross-support window (Sect. 4.1): one pass of a 3x3
// grey-level opening (minimum, then maximum) of the four arm maps
struct SmoothArgs {
    const uchar4 *src[2];
    uchar4 *dst[2];
    uint4 *rec[2];         // dilation pass: records whose L_min and alpha*S follow the new arms
    const float *tables;
    int W, H, rpitch;
};

struct VArgs {
    // per view: the slice as a TMA tile map (dims: disparity within the
    // group, group, x, y; box: the group's 32 disparities plus 4 zero-filled
    // words, of 32 consecutive scan positions)
    CUtensorMap tm[2];
    const uint32_t *sh[2];
    const uchar4 *arms[2];
    unsigned long long *best[2];
    int16_t *disp[2];
    float *cost[2];
    float *vol;            // optional (D, H, W) normalised costs of view `vol_view`
    const int16_t *mask;   // optional: pixels where mask < 0 are written as -1 (vote)
    int *status;           // device status word (a lost tile copy sets a bit)
    int wait_limit;        // mbarrier polls before a tile copy is declared lost
    int skip_copy;         // failure test: arm each tile's barrier but issue no copy
    int tm_rank;           // 4: tm as above; 3: dims (disparity, x, y), box 36 x 1 x 32 at (32 g, x, y)
    int vol_view;
    int W, H, D;           // D: one past the largest disparity of the search (d_min + count)
    int dmin;              // smallest disparity of the search
    int d0, dc, dstride;
    int first, last;       // first / last pass of the d range
    int L1;
    int chunk;             // output rows per block
    int seglog;            // rows per warp segment = 1 << seglog
    float S;
};

struct LrArgs {
    const int16_t *dl, *dr;
    int16_t *out;
    int W, H, tol;
};

} // namespace dco
