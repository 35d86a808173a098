// GB300 (sm_103a) AD-census stereo matcher: kernels and C ABI.
//
// Method: arXiv 2203.02300, Sect. 4 (census + AD cost with adaptive weight,
// Eq. 1; cross-support region aggregation, Eq. 2; winner-take-all, Eq. 3;
// outlier removal by left-right consistency, Sect. 4.3).
//
// Pipeline per pair (one stream, no host round trip):
//   k_pack   RGB -> packed colour words (with the two edge bits of the arm
//            rule's predecessor test) and the grey level, both images
//   k_prep   census (shared-memory grey tile) + the four arms (walks over the
//            packed colours) -> 16-byte records + arm words
//   per pass of dc disparities:
//     k_hagg  Eq. 1 cost in fixed point for every (column, disparity) of a
//             row, prefixes over 16-column segments in shared memory, and
//             the horizontal segment sum of every pixel -> sh slice
//     k_vagg  column prefix of the sh slice (TMA tiles), the vertical sum
//             over the up/down arms (Eq. 2) and the running minimum over
//             the disparities (Eq. 3), merged with the previous passes
//   k_lr     left-right consistency -> disparity map
// Every kernel is launched with programmatic stream serialization and waits
// for its predecessors before its first global access.
// Lanes of a warp hold consecutive disparities of one pixel (pairs of them
// in k_hagg's cost phase): the reference record is a broadcast load, the
// candidates are consecutive records, prefix rows hit distinct banks, and
// the slices are written and read as full 128-byte lines.

#include "kernels.cuh"
#include "dco_stereo.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

namespace dco {

// Programmatic dependent launch: every kernel of the paths is launched with
// programmatic stream serialization, so the launch of a kernel overlaps the
// end of the previous one in the stream.  Before touching global memory a
// block waits until the previous grids have completed and their writes are
// visible.  No block triggers its dependents early: blocks of the next
// kernel parked on free SMs while a multi-pass run's last waves drain made
// those runs slower (1920x1080 in passes of 32: 5.12 against 4.31 ms);
// with the trigger at grid exit the launch latency alone is hidden
// (640x480 D=64: 165 -> 156 us per pair, 320x240 D=32: 46 -> 36.5 us).
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
}


// ------------------------------------------------------------------ k_pack
// RGB (3 bytes per pixel) -> packed 32-bit colour and the integer grey level
// of the census, for both images; four pixels (12 bytes) per thread.
__device__ __forceinline__ uint32_t grey_of(uint32_t c)
{
    return (77u * (c & 0xffu) + 150u * ((c >> 8) & 0xffu) + 29u * ((c >> 16) & 0xffu) + 128u) >> 8;
}

// Colour r | g<<8 | b<<16 spread into three 10-bit fields r | g<<10 | b<<20.
// With K holding tau - 1 + 512 in every field, (E(c) + K - E(p)) keeps each
// field in [1, 1023] (no carry or borrow between fields) and has the field's
// bit 9 set exactly when c_i - p_i + tau - 1 >= 0; the same with c and p
// swapped gives the other side, so every channel has |c_i - p_i| < tau
// exactly when all six bit-9s are set.
constexpr uint32_t kM9 = (1u << 9) | (1u << 19) | (1u << 29);
__device__ __forceinline__ uint32_t spread10(uint32_t c)
{
    return (c & 0xffu) | ((c & 0xff00u) << 2) | ((c & 0xff0000u) << 4);
}
// back to bytes r | g<<8 | b<<16 (bits 30, 31 ignored)
__device__ __forceinline__ uint32_t unspread10(uint32_t e)
{
    return (e & 0xffu) | ((e >> 2) & 0xff00u) | ((e >> 4) & 0xff0000u);
}

// The two bits above the fields of a packed colour: every arm step's colour
// difference to its predecessor must be below tau1 (Sect. 4.1), a property
// of the pixel edge alone, so k_pack stores it once per pixel: bit 30 for
// the edge to the left neighbour, bit 31 for the edge to the one above.
constexpr uint32_t kEdgeL = 1u << 30, kEdgeU = 1u << 31, kColour = 0x3fffffffu;

// all channels within tau of p, given Kp = K - E(p) and pK = E(p) + K
__device__ __forceinline__ bool within(uint32_t ec, uint32_t Kp, uint32_t pK)
{
    return ((ec + Kp) & (pK - ec) & kM9) == kM9;
}

__device__ __forceinline__ uint32_t rgb_at(const uint8_t *rgb, size_t i)
{
    const uint8_t *p = rgb + 3 * i;
    return uint32_t(__ldg(p)) | (uint32_t(__ldg(p + 1)) << 8) | (uint32_t(__ldg(p + 2)) << 16);
}

// k_pack stores every colour spread (the arm walks read each candidate many
// times; the record keeps the bytes) with its two edge bits
__device__ __forceinline__ void pack_body(const PackArgs &a, int q, int img)   // pixels 4q .. 4q+3
{
    const int i0 = 4 * q;
    if (i0 >= a.npx) return;
    const uint8_t *rgb = img ? a.rgb[1] : a.rgb[0];
    uint32_t *rgbx = img ? a.rgbx[1] : a.rgbx[0];
    uint8_t *grey = img ? a.grey[1] : a.grey[0];
    uint32_t c[4];
    if (i0 + 4 <= a.npx && ((reinterpret_cast<uintptr_t>(rgb) & 3u) == 0)) {
        const uint32_t *w = reinterpret_cast<const uint32_t *>(rgb + 3 * (size_t)i0);
        const uint32_t w0 = __ldg(w), w1 = __ldg(w + 1), w2 = __ldg(w + 2);
        c[0] = w0 & 0x00ffffffu;
        c[1] = __funnelshift_r(w0, w1, 24) & 0x00ffffffu;
        c[2] = __funnelshift_r(w1, w2, 16) & 0x00ffffffu;
        c[3] = w2 >> 8;
    } else {
        for (int k = 0; k < 4; k++) {
            const int i = min(i0 + k, a.npx - 1);
            const uint8_t *p = rgb + 3 * (size_t)i;
            c[k] = uint32_t(__ldg(p)) | (uint32_t(__ldg(p + 1)) << 8) | (uint32_t(__ldg(p + 2)) << 16);
        }
    }
    // edge bits: the left neighbour (pixel i - 1 in the same row) and the
    // one above (pixel i - W)
    uint32_t e[4], u[4];
#pragma unroll
    for (int k = 0; k < 4; k++) e[k] = spread10(c[k]);
    const int W = a.W;
    const int up0 = i0 - W;
    if (up0 >= 0 && i0 + 4 <= a.npx && ((reinterpret_cast<uintptr_t>(rgb + 3 * (size_t)up0) & 3u) == 0)) {
        const uint32_t *w = reinterpret_cast<const uint32_t *>(rgb + 3 * (size_t)up0);
        const uint32_t w0 = __ldg(w), w1 = __ldg(w + 1), w2 = __ldg(w + 2);
        u[0] = w0 & 0x00ffffffu;
        u[1] = __funnelshift_r(w0, w1, 24) & 0x00ffffffu;
        u[2] = __funnelshift_r(w1, w2, 16) & 0x00ffffffu;
        u[3] = w2 >> 8;
    } else {
#pragma unroll
        for (int k = 0; k < 4; k++) u[k] = up0 + k >= 0 ? rgb_at(rgb, (size_t)min(up0 + k, a.npx - 1)) : 0u;
    }
    // pixel i0 - 1: the top three bytes of the word before this group (the
    // group starts 4-byte aligned on the aligned path)
    uint32_t prev = 0u;
    if (i0 > 0)
        prev = spread10(((reinterpret_cast<uintptr_t>(rgb) & 3u) == 0)
                            ? __ldg(reinterpret_cast<const uint32_t *>(rgb + 3 * (size_t)i0) - 1) >> 8
                            : rgb_at(rgb, (size_t)(i0 - 1)));
    int x = i0 % W;
    uint32_t out[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const uint32_t Kp = a.k1 - e[k], pK = e[k] + a.k1;
        uint32_t v = e[k];
        if (x > 0 && within(prev, Kp, pK)) v |= kEdgeL;
        if (up0 + k >= 0 && within(spread10(u[k]), Kp, pK)) v |= kEdgeU;
        out[k] = v;
        prev = e[k];
        x = x + 1 == W ? 0 : x + 1;
    }
    if (i0 + 4 <= a.npx) {
        *reinterpret_cast<uint4 *>(rgbx + i0) = make_uint4(out[0], out[1], out[2], out[3]);
        *reinterpret_cast<uint32_t *>(grey + i0) =
            grey_of(c[0]) | (grey_of(c[1]) << 8) | (grey_of(c[2]) << 16) | (grey_of(c[3]) << 24);
    } else {
        for (int k = 0; i0 + k < a.npx; k++) {
            rgbx[i0 + k] = out[k];
            grey[i0 + k] = (uint8_t)grey_of(c[k]);
        }
    }
}

// The same for images in host memory (read over NVLink-C2C, where every
// extra read costs): one thread per block of 4 columns x kRows rows, so the
// row above is read once per block instead of once per row.
template <int kRows>
__device__ __forceinline__ void pack_rows_body(const PackArgs &a, int t, int img)
{
    const int W = a.W, H = a.npx / W;
    const int ngx = (W + 3) >> 2, nby = (H + kRows - 1) / kRows;
    const int band = t / ngx, qx = t - band * ngx;
    if (band >= nby) return;
    const int x0 = 4 * qx, y0 = kRows * band, nx = min(4, W - x0);
    const uint8_t *rgb = img ? a.rgb[1] : a.rgb[0];
    uint32_t *rgbx = img ? a.rgbx[1] : a.rgbx[0];
    uint8_t *grey = img ? a.grey[1] : a.grey[0];
    // rows start 4-byte aligned in the input and 16-byte aligned in the
    // outputs when W is a multiple of 4
    const bool vec = nx == 4 && (W & 3) == 0 && (reinterpret_cast<uintptr_t>(rgb) & 3u) == 0;
    // the four colours of row y at x0 .. x0 + 3 (repeating the last one past
    // the row's end) and the left neighbour (x0 - 1)
    auto load_row = [&](int y, uint32_t (&c)[4], uint32_t &left) {
        const size_t i = (size_t)y * W + x0;
        if (vec) {
            const uint32_t *w = reinterpret_cast<const uint32_t *>(rgb + 3 * i);
            const uint32_t w0 = __ldg(w), w1 = __ldg(w + 1), w2 = __ldg(w + 2);
            c[0] = w0 & 0x00ffffffu;
            c[1] = __funnelshift_r(w0, w1, 24) & 0x00ffffffu;
            c[2] = __funnelshift_r(w1, w2, 16) & 0x00ffffffu;
            c[3] = w2 >> 8;
            left = x0 > 0 ? __ldg(w - 1) >> 8 : 0u;   // the top three bytes of the word before
        } else {
#pragma unroll
            for (int k = 0; k < 4; k++) c[k] = rgb_at(rgb, i + min(k, nx - 1));
            left = x0 > 0 ? rgb_at(rgb, i - 1) : 0u;
        }
    };
    uint32_t up[4] = {0u, 0u, 0u, 0u};   // spread colours of the row above
    if (y0 > 0) {
        uint32_t c[4], l;
        load_row(y0 - 1, c, l);
#pragma unroll
        for (int k = 0; k < 4; k++) up[k] = spread10(c[k]);
    }
#pragma unroll
    for (int r = 0; r < kRows; r++) {
        const int y = y0 + r;
        if (y >= H) break;
        uint32_t c[4], l, e[4], out[4];
        load_row(y, c, l);
#pragma unroll
        for (int k = 0; k < 4; k++) e[k] = spread10(c[k]);
        uint32_t prev = spread10(l);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const uint32_t Kp = a.k1 - e[k], pK = e[k] + a.k1;
            uint32_t v = e[k];
            if (x0 + k > 0 && within(prev, Kp, pK)) v |= kEdgeL;
            if (y > 0 && within(up[k], Kp, pK)) v |= kEdgeU;
            out[k] = v;
            prev = e[k];
            up[k] = e[k];
        }
        const size_t i = (size_t)y * W + x0;
        if (vec) {
            *reinterpret_cast<uint4 *>(rgbx + i) = make_uint4(out[0], out[1], out[2], out[3]);
            *reinterpret_cast<uint32_t *>(grey + i) =
                grey_of(c[0]) | (grey_of(c[1]) << 8) | (grey_of(c[2]) << 16) | (grey_of(c[3]) << 24);
        } else {
            for (int k = 0; k < nx; k++) {
                rgbx[i + k] = out[k];
                grey[i + k] = (uint8_t)grey_of(c[k]);
            }
        }
    }
}

// ------------------------------------------------------------------ k_prep
// One thread per pixel of a 32 x 8 tile.  Census (Sect. 4.2.1) from the grey
// tile with its window halo in shared memory (clamp-to-edge on load); the
// four arms (Sect. 4.1) by walking the packed colours through L1 (arms are
// short on textured input, so no L1-wide halo is staged).  The 9x7 census
// compares four neighbours per SIMD byte comparison.
constexpr int kTX = 32, kTY = 8;
constexpr int kMaxCW = 15, kMaxCH = 15;
constexpr int kGW = 48;   // grey tile row pitch (>= kTX + kMaxCW - 1, multiple of 4)

// 4 flags f_i = [byte_i(w) < byte_i(c4)] -> bits f0 | f1<<1 | f2<<2 | f3<<3.
// Per byte: (w|0x80) - (c&0x7f) never borrows into the next byte, and its top
// bit is clear exactly when the low seven bits compare w < c; the top bits
// of w and c decide the rest.
__device__ __forceinline__ uint32_t lt4(uint32_t w, uint32_t c4, uint32_t c4lo)
{
    const uint32_t x = (w | 0x80808080u) - c4lo;
    const uint32_t lt = ((~w & c4) | (~(w ^ c4) & ~x)) & 0x80808080u;
    return (lt * 0x00204081u) >> 28;
}

template <int CW, int CH>
__device__ __forceinline__ void prep_body(const PrepArgs &a, int bx, int by, int img)
{
    __shared__ __align__(16) uint8_t gs[kTY + kMaxCH - 1][kGW];
    const uint32_t *__restrict__ rgbx = img ? a.rgbx[1] : a.rgbx[0];
    const uint8_t *__restrict__ grey = img ? a.grey[1] : a.grey[0];
    const int W = a.W, H = a.H;
    const int cw = CW ? CW : a.cw, ch = CH ? CH : a.ch;
    const int rx = cw / 2, ry = ch / 2;
    const int x0 = bx * kTX, y0 = by * kTY;
    const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;   // 1-D block of kTX x kTY threads
    for (int r = ty; r < kTY + 2 * ry; r += kTY) {
        const int y = min(max(y0 - ry + r, 0), H - 1);
        for (int c = tx; c < kTX + 2 * rx; c += kTX) {
            const int x = min(max(x0 - rx + c, 0), W - 1);
            gs[r][c] = __ldg(grey + (size_t)y * W + x);
        }
    }
    __syncthreads();
    const int x = x0 + tx, y = y0 + ty;
    if (x >= W || y >= H) return;

    // census: bit k = [Y(n) < Y(p)], window row-major, centre skipped
    const uint32_t yc = gs[ty + ry][tx + rx];
    unsigned long long bits = 0ull;
    if (CW == 9 && CH == 7) {
        const uint32_t c4 = yc * 0x01010101u, c4lo = c4 & 0x7f7f7f7fu;
        const int al = tx & ~3, sh = 8 * (tx & 3);
        int k = 0;
#pragma unroll
        for (int dy = 0; dy < 7; dy++) {
            const uint32_t *row = reinterpret_cast<const uint32_t *>(&gs[ty + dy][al]);
            const uint32_t a0 = row[0], a1 = row[1], a2 = row[2];
            const uint32_t w0 = __funnelshift_r(a0, a1, sh);   // bytes dx 0..3
            const uint32_t w1 = __funnelshift_r(a1, a2, sh);   // bytes dx 4..7
            const uint32_t b8 = (__funnelshift_r(a2, 0u, sh) & 0xffu) < yc ? 1u : 0u;   // dx 8
            const uint32_t f0 = lt4(w0, c4, c4lo), f1 = lt4(w1, c4, c4lo);
            uint32_t rowbits;
            int nb;
            if (dy == 3) {   // centre row: dx 4 is the centre itself
                rowbits = f0 | ((f1 >> 1) << 4) | (b8 << 7);
                nb = 8;
            } else {
                rowbits = f0 | (f1 << 4) | (b8 << 8);
                nb = 9;
            }
            bits |= (unsigned long long)rowbits << k;
            k += nb;
        }
    } else {
        int k = 0;
        for (int dy = 0; dy < ch; dy++) {
            for (int dx = 0; dx < cw; dx++) {
                if (dy == ry && dx == rx) continue;
                if (gs[ty + dy][tx + dx] < yc) bits |= 1ull << k;
                k++;
            }
        }
    }

    // arms: largest k <= L1 whose steps all pass the double threshold
    const size_t i = (size_t)y * W + x;
    const uint32_t praw = __ldg(rgbx + i);   // colours are stored spread (k_pack), with edge bits
    const uint32_t p = praw & kColour;
    const int L1 = a.L1, L2 = a.L2;
    // K = t - 1 + 512 in each 10-bit field, t = min(tau, 256): the field of
    // E(c) + K - E(q) has bit 9 set exactly when c - q > -t, and with t = 256
    // every pair passes (a threshold of 256 or more never stops an arm).
    // Up to L2 a step is tested against p with tau1; beyond L2 against p
    // with min(tau1, tau2) (both must hold).  The test against the step's
    // predecessor (tau1) is the edge bit k_pack stored: the candidate's own
    // for walks right and down (its edge towards p), the predecessor's for
    // walks left and up.
    auto kfield = [](int tau) { return 0x00100401u * (uint32_t)(min(tau, 256) + 511); };
    const uint32_t k1 = kfield(a.tau1), k2 = kfield(min(a.tau1, a.tau2));
    const uint32_t K1p = k1 - p, pK1 = p + k1, K2p = k2 - p, pK2 = p + k2;
    auto pass = [](uint32_t c, uint32_t Kp, uint32_t pK, uint32_t ew, uint32_t bit) {
        return ((((c + Kp) & (pK - c)) & kM9 | (ew & bit)) == (kM9 | bit));
    };
    // the first kArmBatch candidates of all four directions are loaded at
    // once (in-image addresses only), so a typical pixel pays one load latency
    constexpr int kArmBatch = 2;
    int arm[4];
    uint32_t cand[4][kArmBatch];
    int lim[4];
    ptrdiff_t step[4];
#pragma unroll
    for (int e = 0; e < 4; e++) {
        const int room = e == 0 ? x : (e == 1 ? W - 1 - x : (e == 2 ? y : H - 1 - y));
        step[e] = e == 0 ? -1 : (e == 1 ? 1 : (e == 2 ? -(ptrdiff_t)W : (ptrdiff_t)W));
        lim[e] = min(L1, room);
#pragma unroll
        for (int u = 0; u < kArmBatch; u++)
            cand[e][u] = u < lim[e] ? __ldg(rgbx + i + (u + 1) * step[e]) : 0u;
    }
#pragma unroll
    for (int e = 0; e < 4; e++) {
        const uint32_t bit = e < 2 ? kEdgeL : kEdgeU;
        const bool own = e & 1;   // right, down: the candidate's own edge bit
        uint32_t prev = praw;     // left, up: the predecessor's (p itself before step 1)
        int n = 0;
        bool open = true;
#pragma unroll
        for (int u = 0; u < kArmBatch; u++) {
            const int j = u + 1;
            const bool far = j > L2;
            const uint32_t c = cand[e][u];
            if (open && j <= lim[e] && pass(c, far ? K2p : K1p, far ? pK2 : pK1, own ? c : prev, bit)) {
                n = j;
                prev = c;
            } else {
                open = false;
            }
        }
        // longer arms: one candidate at a time, up to L2 then beyond
        if (open) {
            const uint32_t *q = rgbx + i + (ptrdiff_t)n * step[e];
            int j = n + 1;
            if (own) {
                for (const int l = min(lim[e], L2); j <= l; j++) {
                    q += step[e];
                    const uint32_t c = __ldg(q);
                    if (!pass(c, K1p, pK1, c, bit)) { open = false; break; }
                }
                if (open) {
                    for (; j <= lim[e]; j++) {
                        q += step[e];
                        const uint32_t c = __ldg(q);
                        if (!pass(c, K2p, pK2, c, bit)) break;
                    }
                }
            } else {
                for (const int l = min(lim[e], L2); j <= l; j++) {
                    q += step[e];
                    const uint32_t c = __ldg(q);
                    if (!pass(c, K1p, pK1, prev, bit)) { open = false; break; }
                    prev = c;
                }
                if (open) {
                    for (; j <= lim[e]; j++) {
                        q += step[e];
                        const uint32_t c = __ldg(q);
                        if (!pass(c, K2p, pK2, prev, bit)) break;
                        prev = c;
                    }
                }
            }
            n = j - 1;
        }
        arm[e] = n;
    }
    const int lmin = min(min(arm[0], arm[1]), min(arm[2], arm[3]));
    const float alphaS = __ldg(a.tables + kTabAD + kTabCen + lmin);
    const uint32_t colour = unspread10(p) | (uint32_t(lmin) << 24);
    (img ? a.rec[1] : a.rec[0])[(size_t)y * a.rpitch + x] =
        make_uint4((uint32_t)bits, (uint32_t)(bits >> 32), colour, __float_as_uint(alphaS));
    const size_t pe = (size_t)y * 2 * a.phw + (size_t)(x & 1) * a.phw + (x >> 1);
    (img ? a.cen[1] : a.cen[0])[pe] = make_uint2((uint32_t)bits, (uint32_t)(bits >> 32));
    (img ? a.col[1] : a.col[0])[pe] = colour;
    (img ? a.arms[1] : a.arms[0])[i] = make_uchar4((uint8_t)arm[0], (uint8_t)arm[1], (uint8_t)arm[2], (uint8_t)arm[3]);
}

// --------------------------------------------------------------- k_smooth
// Smooth cross-support window (Sect. 4.1, morphological processing): the
// opening of each arm map is a 3x3 minimum (kMax = false) followed by a 3x3
// maximum (kMax = true), windows cut to the image.  An opening never
// lengthens an arm, so arms stay inside the image and <= L1.  The maximum
// pass also rewrites the record's L_min and alpha(L_min)*S (Eq. 1).
template <bool kMax>
__device__ __forceinline__ void smooth_body(const SmoothArgs &a, int i, int img)
{
    if (i >= a.W * a.H) return;
    const int x = i % a.W, y = i / a.W;
    const uchar4 *src = img ? a.src[1] : a.src[0];
    int v[4] = {kMax ? 0 : 255, kMax ? 0 : 255, kMax ? 0 : 255, kMax ? 0 : 255};
    for (int yy = max(0, y - 1); yy <= min(a.H - 1, y + 1); yy++)
        for (int xx = max(0, x - 1); xx <= min(a.W - 1, x + 1); xx++) {
            const uchar4 q = src[(size_t)yy * a.W + xx];
            const int c[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; k++) v[k] = kMax ? max(v[k], c[k]) : min(v[k], c[k]);
        }
    (img ? a.dst[1] : a.dst[0])[i] = make_uchar4((uint8_t)v[0], (uint8_t)v[1], (uint8_t)v[2], (uint8_t)v[3]);
    uint4 *rec = img ? a.rec[1] : a.rec[0];
    if (kMax && rec) {
        const int lmin = min(min(v[0], v[1]), min(v[2], v[3]));
        uint4 *r = rec + (size_t)y * a.rpitch + x;
        r->z = (r->z & 0x00ffffffu) | (uint32_t(lmin) << 24);
        r->w = __float_as_uint(__ldg(a.tables + kTabAD + kTabCen + lmin));
    }
}

// ------------------------------------------------------------------ k_hagg
// Block = one row segment of one reference view for one group of 32
// disparities.  Stage 0 copies (cp.async) the tables, the reference records
// of the prefix range [xa, xb) (the output columns plus an L1 reach on both
// sides), the candidate records of the whole group (census and colour apart,
// even and odd candidate indices apart) and the output columns' arms into
// shared memory.  Then:
//   A. each half-warp walks a segment of 16 columns; lane j of the half holds
//      the disparity pair (dlo + 2j, dlo + 2j + 1): Eq. 1 costs rounded to
//      fixed point, local inclusive prefixes into P[x - xa][d - dlo].  The
//      candidate of d + 1 at column x + 1 is the candidate of d at x (the
//      other way round in the right-reference view), so each column step
//      loads one new candidate record for two evaluations;
//   B. the exclusive prefix of the segment totals (segment offsets);
//   C. every output column xo: S_H = F(xo + r) - F(xo - l - 1) (the
//      horizontal part of Eq. 2), F the row prefix: the difference of the
//      local prefixes plus the difference of their segments' offsets.
// Unsigned wrap-around makes the differences exact segment sums.
constexpr int kTabBytes = (kTabAD + kTabCen) * 4;

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

constexpr int kWaitLimit = 1 << 22;   // mbarrier polls before a copy is declared lost
constexpr int kTestWaitLimit = 64;    // the same, under the lost-copy failure test
constexpr int kStatusCopyTimeout = 1; // status word: a copy (k_hagg staging, k_vagg tiles) did not complete
constexpr int kStatusAlign = 2;       // status word: shared memory not aligned for the tile copies

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}
// bounded wait for the phase of the given parity to complete: false after
// `limit` polls without completion
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit)
{
    for (int i = 0; i < limit; i++) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (ok) return true;
    }
    return false;
}
// bulk copy of n bytes (a multiple of 16; both addresses 16-byte aligned)
// from global memory to shared memory, completing on mbarrier `bar`
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t n, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(n), "r"(bar)
                 : "memory");
}

// byte offsets of the H block's shared-memory regions.  Candidate indices
// run over [0, len + 31); index i sits at position i >> 1 of the even (i & 1
// = 0) or odd array, hh positions each.  The arrays arrive by bulk copies
// that start on 16-byte boundaries of the candidate planes, so each half has
// room for the alignment shift: census halves hhc entries (up to one more
// than hh, even), colour halves hhk (up to three more, a multiple of 4), the
// arms up to three entries more.
struct HSmem {
    int ref, oth, hh, hhc, hhk, col, arm, p, t, total;
    __host__ __device__ HSmem(int len, int chunk, int nw)
    {
        ref = kTabBytes;
        oth = ref + len * 16;                   // census: uint2 [2][hhc]; then the segment offsets
        hh = (len + 33) / 2;
        hhc = (hh + 3) & ~1;
        hhk = (hh + 9) & ~3;
        col = oth + hhc * 16;                   // colour: uint32 [2][hhk]
        arm = col + hhk * 8;
        p = arm + ((chunk + 9) & ~3) * 4 + 128; // one zero row in front: P[-1]
        t = p + len * 128;
        total = t + 2 * nw * 128;               // segment totals [2 nw][32]
    }
};

// Phase C of a horizontal pass: every output column c (n_out of them,
// prefix index base + c): S_H = F(c + r) - F(c - l - 1), F the prefix of the
// costs along the scan.  P holds prefixes local to segments of 1 << kSegLog
// positions and OFF the exclusive prefix of the segment totals, so
// F(x) = OFF[x >> kSegLog] + P(x) and F(-1) = 0 (the zero row in front of P,
// segment 0 whose offset is 0); no pass over P adds offsets.  Each
// quarter-warp takes one column, lane j of the quarter the disparities
// 4j .. 4j + 3 of the group (16-byte loads and stores, one 128-byte prefix
// row per quarter).  Unsigned wrap-around makes the differences exact.
template <int kSegLog>
__device__ __forceinline__ void hagg_out_quads(const uint32_t *P, const uint32_t *OFF, const uchar4 *sarm, int n_out,
                                               int base, uint32_t *o, size_t ds)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int l8 = lane & 7;
    const uint4 *P4 = reinterpret_cast<const uint4 *>(P) + l8;
    const uint4 *F4 = reinterpret_cast<const uint4 *>(OFF) + l8;
    uint4 *o4 = reinterpret_cast<uint4 *>(o) + l8;
    const size_t ds4 = ds / 4;
    auto column = [&](int i) -> uint4 {
        const uchar4 am = sarm[i];
        const int hi = base + i + am.y, lo = base + i - am.x - 1;   // lo >= -1
        const uint4 a = P4[hi * 8], b = P4[lo * 8];
        uint4 v = make_uint4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
        const int sh = hi >> kSegLog, sl = max(lo, 0) >> kSegLog;
        if (sh != sl) {   // the arm interval crosses segment boundaries
            const uint4 fh = F4[sh * 8], fl = F4[sl * 8];
            v.x += fh.x - fl.x;
            v.y += fh.y - fl.y;
            v.z += fh.z - fl.z;
            v.w += fh.w - fl.w;
        }
        return v;
    };
    int i = 4 * warp + (lane >> 3);
    const int step = 4 * nw;
    for (; i + step < n_out; i += 2 * step) {
        const uint4 v0 = column(i), v1 = column(i + step);
        o4[(size_t)i * ds4] = v0;
        o4[(size_t)(i + step) * ds4] = v1;
    }
    if (i < n_out) o4[(size_t)i * ds4] = column(i);
}

// Phases B and C of a horizontal pass (k_vcost, k_hvote) whose warps each
// scanned one segment of 1 << kSegLog positions: P holds every warp's local
// inclusive prefix of its segment, T the segment totals (visible after a
// barrier).
//   B. T is replaced by the exclusive prefix of the totals (segment offsets);
//   C. hagg_out_quads with those offsets.
template <int kSegLog>
__device__ __forceinline__ void hagg_tail(const uint32_t *P, uint32_t *T, const uchar4 *sarm, int n_out, int base,
                                          uint32_t *o, size_t ds)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t offs = 0;
#pragma unroll 4
    for (int w = 0; w < warp; w++) offs += T[w * 32 + lane];
    __syncthreads();
    T[warp * 32 + lane] = offs;
    __syncthreads();
    hagg_out_quads<kSegLog>(P, T, sarm, n_out, base, o, ds);
}

// Phase A of k_hagg for one half-warp segment [sa, sb) (relative to xa) of
// view kView.  Lane j of the half (hl) holds the disparities da = dlo + 2 hl
// and da + 1, the prefixes run_a, run_b.  The candidate index of the record
// loaded new at column x is x + nb (odd at even x): view 0 pairs it with da
// and the previous one with da + 1, view 1 the other way round.  A match
// outside the image costs 1 (Sint): view 0 needs x >= va / vb, view 1 x < va / vb.
template <int kView>
__device__ __forceinline__ void hagg_costs(const uint4 *sref, const uint2 *cenE, const uint2 *cenO,
                                           const uint32_t *colE, const uint32_t *colO, const float *sTA,
                                           const float *sTC, uint32_t *P, int sa, int sb, int hl, int va, int vb,
                                           float Sf, uint32_t Sint, uint32_t &run_a, uint32_t &run_b)
{
    const int nb = kView ? 1 + 2 * hl : 31 - 2 * hl;
    const int p0 = (sa + nb - 1) >> 1;
    const uint2 *cE = cenE + p0 + 1, *cO = cenO + p0;   // new records at odd / even steps
    const uint32_t *kE = colE + p0 + 1, *kO = colO + p0;
    uint2 pc = cenE[p0];
    uint32_t pk = colE[p0];
    uint2 *Pp = reinterpret_cast<uint2 *>(P) + hl;
    auto cost = [&](const uint4 &pr, float av, float sav, uint2 c, uint32_t col) -> uint32_t {
        const int h = __popc(pr.x ^ c.x) + __popc(pr.y ^ c.y);
        const int k = (int)__dp4a(__vabsdiffu4(pr.z, col), 0x00010101u, 0u);
        return __float2uint_rn(fmaf(av, sTA[k], sav * sTC[h]));
    };
    auto step = [&](int x, uint2 nc, uint32_t nk) {
        const uint4 pr = sref[x];
        const float av = __uint_as_float(pr.w), sav = Sf - av;
        const uint32_t qa = kView ? cost(pr, av, sav, pc, pk) : cost(pr, av, sav, nc, nk);
        const uint32_t qb = kView ? cost(pr, av, sav, nc, nk) : cost(pr, av, sav, pc, pk);
        run_a += (kView ? x < va : x >= va) ? qa : Sint;
        run_b += (kView ? x < vb : x >= vb) ? qb : Sint;
        Pp[x * 16] = make_uint2(run_a, run_b);
        pc = nc;
        pk = nk;
    };
    if (sb - sa == 16) {
#pragma unroll
        for (int k = 0; k < 8; k++) {
            step(sa + 2 * k, cO[k], kO[k]);
            step(sa + 2 * k + 1, cE[k], kE[k]);
        }
    } else {
        for (int k = 0; sa + 2 * k < sb; k++) {
            step(sa + 2 * k, cO[k], kO[k]);
            if (sa + 2 * k + 1 < sb) step(sa + 2 * k + 1, cE[k], kE[k]);
        }
    }
}

__device__ __forceinline__ void hagg_body(const HArgs &a, int bx, int by, int bz)
{
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int W = a.W, L1 = a.L1;
    const int y = by;
    const int view = bz / a.ngroups, g = bz % a.ngroups;
    const int xs = bx * a.chunk, xe = min(W, xs + a.chunk);
    const int xa = max(0, xs - L1), xb = min(W, xe + L1), len = xb - xa;
    const HSmem L(len, a.chunk, nw);
    float *sTA = reinterpret_cast<float *>(smem_raw);
    float *sTC = sTA + kTabAD;
    uint4 *sref = reinterpret_cast<uint4 *>(smem_raw + L.ref);
    uint2 *scen = reinterpret_cast<uint2 *>(smem_raw + L.oth);       // candidate census [2][hhc]
    uint32_t *scol = reinterpret_cast<uint32_t *>(smem_raw + L.col); // candidate colour + Lmin [2][hhk]
    uchar4 *sarm = reinterpret_cast<uchar4 *>(smem_raw + L.arm);
    uint32_t *P = reinterpret_cast<uint32_t *>(smem_raw + L.p);   // [len][32], P[-1] = 0
    uint32_t *T = reinterpret_cast<uint32_t *>(smem_raw + L.t);   // [2 nw][32]
    if (threadIdx.x < 32) P[(int)threadIdx.x - 32] = 0u;

    // first disparity of this group
    const int dlo = a.d0 + 32 * g;
    // candidate index i <-> column olo + i, i in [0, len + 31): every
    // disparity of the 32-wide group (the costs of dead disparities are
    // computed from whatever the shared words hold and never read)
    const int olo = view ? xa + dlo : xa - dlo - 31;
    const uint4 *rref = (view ? a.rec[1] : a.rec[0]) + (size_t)y * a.rpitch;

    // ---- 0: stage by bulk copies, issued by one thread on one mbarrier:
    // the tables, the reference records, the arms and the candidates.  The
    // even-index candidates i = 2m are the columns olo + 2m, entry
    // (olo >> 1) + m of one half of the other view's plane row, the odd ones
    // olo + 1 + 2m of the other half; only the in-image columns are copied
    // (the others cost 1 whatever they hold).  Each copy starts on the 16-byte
    // boundary at or below its first entry, and candidate m of a half sits at
    // shared position o + m, o (0-3) chosen so the copy's destination is
    // 16-byte aligned too.
    __shared__ __align__(8) unsigned long long hbar_s;
    __shared__ int hoff_s[5];   // the halves' shared offsets o, then the lost flag
    const uint32_t hbar = (uint32_t)__cvta_generic_to_shared(&hbar_s);
    const size_t ga = (size_t)y * W + xs, gas = ga & ~(size_t)3;
    if (threadIdx.x == 0) {
        struct Half {
            int base, mlo, mhi;   // plane entry of m = 0 (may be negative), in-image m range
        };
        auto cand_half = [&](int c0) {   // the candidates c0 + 2m, m < hh
            Half h;
            h.base = (c0 & 1) * a.phw + (c0 >> 1);
            h.mlo = max(0, (1 - c0) >> 1);          // first m with c0 + 2m >= 0
            h.mhi = min(L.hh, (W - c0 + 1) >> 1);   // first m with c0 + 2m >= W
            return h;
        };
        const Half hE = cand_half(olo), hO = cand_half(olo + 1);
        // q entries per 16 bytes: the copy starts `shift` entries below the
        // first in-image one; o makes (o + mlo - shift) a multiple of q
        auto shift = [](const Half &h, int q) { return h.mlo < h.mhi ? (h.base + h.mlo) & (q - 1) : 0; };
        auto offs = [&](const Half &h, int q) { return (shift(h, q) - h.mlo) & (q - 1); };
        auto count = [&](const Half &h, int q) {
            return h.mlo < h.mhi ? (uint32_t)(h.mhi - h.mlo + shift(h, q) + q - 1) & ~(uint32_t)(q - 1) : 0u;
        };
        const uint2 *cpl = (view ? a.cen[0] : a.cen[1]) + (size_t)y * 2 * a.phw;
        const uint32_t *kpl = (view ? a.col[0] : a.col[1]) + (size_t)y * 2 * a.phw;
        const uint32_t nA = (uint32_t)(xe - xs + (int)(ga - gas) + 3) & ~3u;
        const uint32_t nCE = count(hE, 2), nCO = count(hO, 2), nKE = count(hE, 4), nKO = count(hO, 4);
        const int oCE = offs(hE, 2), oCO = offs(hO, 2), oKE = offs(hE, 4), oKO = offs(hO, 4);
        mbar_init(hbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        mbar_expect_tx(hbar, (uint32_t)kTabBytes + 16u * (uint32_t)len + 8u * (nCE + nCO) + 4u * (nKE + nKO) + 4u * nA);
        if (!a.skip_copy) {   // (the failure test arms the barrier and issues nothing)
            bulk_g2s(smem_raw, a.tables, kTabBytes, hbar);
            bulk_g2s(sref, rref + xa, 16u * (uint32_t)len, hbar);
            bulk_g2s(sarm, (view ? a.arms[1] : a.arms[0]) + gas, 4u * nA, hbar);
            if (nCE) bulk_g2s(scen + oCE + hE.mlo - shift(hE, 2), cpl + hE.base + hE.mlo - shift(hE, 2), 8u * nCE, hbar);
            if (nCO)
                bulk_g2s(scen + L.hhc + oCO + hO.mlo - shift(hO, 2), cpl + hO.base + hO.mlo - shift(hO, 2), 8u * nCO, hbar);
            if (nKE) bulk_g2s(scol + oKE + hE.mlo - shift(hE, 4), kpl + hE.base + hE.mlo - shift(hE, 4), 4u * nKE, hbar);
            if (nKO)
                bulk_g2s(scol + L.hhk + oKO + hO.mlo - shift(hO, 4), kpl + hO.base + hO.mlo - shift(hO, 4), 4u * nKO, hbar);
        }
        hoff_s[0] = oCE;
        hoff_s[1] = oCO;
        hoff_s[2] = oKE;
        hoff_s[3] = oKO;
        const bool ok = mbar_wait(hbar, 0u, a.wait_limit);
        if (!ok) {   // report, and wait (bounded) once more before the block's shared memory is released
            if (a.status) atomicOr(a.status, kStatusCopyTimeout);
            mbar_wait(hbar, 0u, a.wait_limit);
        }
        hoff_s[4] = !ok;
    }
    __syncthreads();
    if (hoff_s[4]) return;
    const uint2 *cenE = scen + hoff_s[0], *cenO = scen + L.hhc + hoff_s[1];
    const uint32_t *colE = scol + hoff_s[2], *colO = scol + L.hhk + hoff_s[3];
    const uchar4 *sarm0 = sarm + (ga - gas);   // arm of output column xs

    // ---- A: costs and local prefixes of this half-warp's segment
    const int half = lane >> 4, hl = lane & 15;
    const int s = 2 * warp + half;
    const int sa = 16 * s, sb = min(len, sa + 16);
    const int da = dlo + 2 * hl;
    // columns x (relative to xa) whose match x -/+ d lies in the image
    const int va = view ? W - xa - da : da - xa, vb = view ? va - 1 : va + 1;
    uint32_t run_a = 0, run_b = 0;
    if (sa < len) {
        if (view)
            hagg_costs<1>(sref, cenE, cenO, colE, colO, sTA, sTC, P, sa, sb, hl, va, vb, a.S, a.Sint, run_a, run_b);
        else
            hagg_costs<0>(sref, cenE, cenO, colE, colO, sTA, sTC, P, sa, sb, hl, va, vb, a.S, a.Sint, run_a, run_b);
    }
    reinterpret_cast<uint2 *>(T + s * 32)[hl] = make_uint2(run_a, run_b);
    __syncthreads();

    // ---- B: exclusive offsets of the segments holding columns (lane =
    // disparity), written over the candidate records, which are no longer read
    uint32_t *OFF = reinterpret_cast<uint32_t *>(smem_raw + L.oth);   // [ceil(len / 16)][32]
    if (32 * warp < len) {
        uint32_t offs = 0;
#pragma unroll 4
        for (int s2 = 0; s2 < 2 * warp; s2++) offs += T[s2 * 32 + lane];
        OFF[2 * warp * 32 + lane] = offs;
        if (32 * warp + 16 < len) OFF[(2 * warp + 1) * 32 + lane] = offs + T[2 * warp * 32 + lane];
    }
    __syncthreads();

    // ---- C
    hagg_out_quads<4>(P, OFF, sarm0, xe - xs, xs - xa,
                      (view ? a.sh[1] : a.sh[0]) + ((size_t)y * W + xs) * a.dstride + g * 32, a.dstride);
}

// ---------------------------------------------------------------- k_vcost
// The other aggregation order, first pass: Eq. 1 costs and their vertical
// segment sums S_V(q, d) over q's vertical arm.  Block = one column x (a
// chunk of rows) of one reference view for one group of 32 disparities;
// lane = disparity.  The reference records of the column are staged in
// shared memory; the candidates of each row (32 neighbouring records of the
// other view's row) are read straight from the record rows.  Then the
// phases of a horizontal pass along the column: local prefixes over warp
// segments of 32 rows, segment offsets, segment sums (hagg_tail, with the
// up / down arms), written to the same slice layout.
struct CSmem {
    int ref, arm, p, t, total;
    __host__ __device__ CSmem(int len, int chunk, int nw)
    {
        ref = kTabBytes;
        arm = ref + len * 16;
        p = arm + (chunk + 3) / 4 * 16 + 128;   // one zero row in front: P[-1]
        t = p + len * 128;
        total = t + nw * 128;
    }
};

__device__ __forceinline__ void vcost_body(const HArgs &a, int bx, int by, int bz)
{
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int W = a.W, H = a.H, L1 = a.L1;
    const int x = bx;
    const int view = bz / a.ngroups, g = bz % a.ngroups;
    const int ys = by * a.chunk, ye = min(H, ys + a.chunk);
    const int ya = max(0, ys - L1), yb = min(H, ye + L1), len = yb - ya;
    const CSmem L(len, a.chunk, nw);
    const float *sTA = reinterpret_cast<const float *>(smem_raw);
    const float *sTC = sTA + kTabAD;
    uint4 *sref = reinterpret_cast<uint4 *>(smem_raw + L.ref);
    uchar4 *sarm = reinterpret_cast<uchar4 *>(smem_raw + L.arm);   // (up, down) of the output rows
    uint32_t *P = reinterpret_cast<uint32_t *>(smem_raw + L.p);    // [len][32], P[-1] = 0
    uint32_t *T = reinterpret_cast<uint32_t *>(smem_raw + L.t);
    const uint4 *rref = view ? a.rec[1] : a.rec[0];   // padded rows, pitch rpitch
    const uint4 *roth = view ? a.rec[0] : a.rec[1];
    const uchar4 *aref = view ? a.arms[1] : a.arms[0];

    for (int i = threadIdx.x; i < kTabBytes / 16; i += blockDim.x)
        cp_async16(smem_raw + 16 * i, reinterpret_cast<const uint8_t *>(a.tables) + 16 * i);
    for (int i = threadIdx.x; i < len; i += blockDim.x) cp_async16(sref + i, rref + (size_t)(ya + i) * a.rpitch + x);
    for (int i = threadIdx.x; i < ye - ys; i += blockDim.x) {
        const uchar4 am = aref[(size_t)(ys + i) * W + x];
        sarm[i] = make_uchar4(am.z, am.w, 0, 0);   // backward = up, forward = down
    }
    if (threadIdx.x < 32) P[(int)threadIdx.x - 32] = 0u;
    cp_async_wait_all();
    __syncthreads();

    const int dlo = a.d0 + 32 * g;
    const int dhi = min(min(a.d0 + a.dc, a.D), dlo + 32) - 1;
    const int d = dlo + lane;
    const int dd = d <= dhi ? d : dlo;                // dead lanes read a real candidate, results unused
    const int xo = view ? x + dd : x - dd;            // candidate column, -255 .. W + 254 (padded rows)
    const bool outside = xo < 0 || xo >= W;           // match outside the image: cost 1
    const uint4 *cand = roth + xo;
    const float Sf = a.S;
    const uint32_t Sint = a.Sint;

    // ---- A: costs down this warp's segment of rows, local prefix
    const int sa = warp * kHSegCost, sb = min(len, sa + kHSegCost);   // rows relative to ya
    uint32_t run = 0;
    int u = sa;
    for (; u + 4 <= sb; u += 4) {
        uint4 po[4];
#pragma unroll
        for (int k = 0; k < 4; k++) po[k] = __ldg(cand + (size_t)(ya + u + k) * a.rpitch);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const uint4 pr = sref[u + k];
            const int hm = __popc(pr.x ^ po[k].x) + __popc(pr.y ^ po[k].y);
            const int kk = (int)__dp4a(__vabsdiffu4(pr.z, po[k].z), 0x00010101u, 0u);
            const float av = __uint_as_float(pr.w);
            const uint32_t q = __float2uint_rn(fmaf(av, sTA[kk], (Sf - av) * sTC[hm]));
            run += outside ? Sint : q;
            P[(u + k) * 32 + lane] = run;
        }
    }
    for (; u < sb; u++) {
        const uint4 po = __ldg(cand + (size_t)(ya + u) * a.rpitch);
        const uint4 pr = sref[u];
        const int hm = __popc(pr.x ^ po.x) + __popc(pr.y ^ po.y);
        const int kk = (int)__dp4a(__vabsdiffu4(pr.z, po.z), 0x00010101u, 0u);
        const float av = __uint_as_float(pr.w);
        const uint32_t q = __float2uint_rn(fmaf(av, sTA[kk], (Sf - av) * sTC[hm]));
        run += outside ? Sint : q;
        P[u * 32 + lane] = run;
    }
    T[warp * 32 + lane] = run;
    __syncthreads();
    // consecutive output rows are one slice row (W * dstride words) apart
    static_assert(kHSegCost == 1 << 5, "k_vcost segments: 32 rows per warp");
    hagg_tail<5>(P, T, sarm, ye - ys, ys - ya, (view ? a.sh[1] : a.sh[0]) + ((size_t)ys * W + x) * a.dstride + g * 32,
                 (size_t)W * a.dstride);
}

// ---------------------------------------------------------------- k_hvote
// Horizontal pass of the parallax optimisation (Sect. 4.3, Eq. 4): block =
// (row, group of 32 disparities), lane = disparity, local prefixes over warp
// segments of 64 columns of the indicator [disp(x, y) == d] of the map being
// voted on (-1 matches no d), then the output phase of the horizontal passes,
// so S_H holds the number of pixels of each horizontal segment that vote for
// d.  A local prefix counts at most 64 columns, so P keeps it in one byte
// per disparity (32 bytes per column): a quarter of the 4-byte prefix rows
// of the cost pass, so that more blocks fit an SM.
struct HVSmem {
    int disp, arm, p, t, total;
    __host__ __device__ HVSmem(int len, int chunk, int nw)
    {
        disp = 0;
        arm = (len * 2 + 15) / 16 * 16;
        p = arm + (chunk + 3) / 4 * 16 + 32;    // one zero row in front: P[-1]
        t = p + (len * 32 + 15) / 16 * 16;
        total = t + nw * 128;
    }
};

// The output phase of k_hvote: as hagg_out_quads, with byte prefixes (each
// lane of a quarter-warp reads the four counts of its disparities 4j .. 4j + 3
// as one word and widens them; unsigned wrap-around keeps the differences
// exact once the segment offsets are added).
template <int kSegLog>
__device__ __forceinline__ void hvote_out_quads(const uint8_t *P, const uint32_t *OFF, const uchar4 *sarm,
                                                int n_out, int base, uint32_t *o, size_t ds)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int l8 = lane & 7;
    const uint32_t *P4 = reinterpret_cast<const uint32_t *>(P) + l8;   // rows of 8 words
    const uint4 *F4 = reinterpret_cast<const uint4 *>(OFF) + l8;
    uint4 *o4 = reinterpret_cast<uint4 *>(o) + l8;
    const size_t ds4 = ds / 4;
    auto column = [&](int i) -> uint4 {
        const uchar4 am = sarm[i];
        const int hi = base + i + am.y, lo = base + i - am.x - 1;   // lo >= -1
        const uint32_t a = P4[hi * 8], b = P4[lo * 8];
        uint4 v = make_uint4((a & 0xffu) - (b & 0xffu), ((a >> 8) & 0xffu) - ((b >> 8) & 0xffu),
                             ((a >> 16) & 0xffu) - ((b >> 16) & 0xffu), (a >> 24) - (b >> 24));
        const int sh = hi >> kSegLog, sl = max(lo, 0) >> kSegLog;
        if (sh != sl) {   // the arm interval crosses segment boundaries
            const uint4 fh = F4[sh * 8], fl = F4[sl * 8];
            v.x += fh.x - fl.x;
            v.y += fh.y - fl.y;
            v.z += fh.z - fl.z;
            v.w += fh.w - fl.w;
        }
        return v;
    };
    int i = 4 * warp + (lane >> 3);
    const int step = 4 * nw;
    for (; i + step < n_out; i += 2 * step) {
        const uint4 v0 = column(i), v1 = column(i + step);
        o4[(size_t)i * ds4] = v0;
        o4[(size_t)(i + step) * ds4] = v1;
    }
    if (i < n_out) o4[(size_t)i * ds4] = column(i);
}

__device__ __forceinline__ void hvote_body(const HVArgs &a, int bx, int by, int bz)
{
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int W = a.W, L1 = a.L1;
    const int y = by, g = bz;
    const int xs = bx * a.chunk, xe = min(W, xs + a.chunk);
    const int xa = max(0, xs - L1), xb = min(W, xe + L1), len = xb - xa;
    const HVSmem L(len, a.chunk, nw);
    int16_t *sd = reinterpret_cast<int16_t *>(smem_raw + L.disp);
    uchar4 *sarm = reinterpret_cast<uchar4 *>(smem_raw + L.arm);
    uint8_t *P = smem_raw + L.p;                                   // [len][32] bytes, P[-1] = 0
    uint32_t *T = reinterpret_cast<uint32_t *>(smem_raw + L.t);   // [nw][32]
    if (threadIdx.x < 32) P[(int)threadIdx.x - 32] = 0;
    const int16_t *drow = a.disp + (size_t)y * W;
    const uchar4 *aref = a.arms + (size_t)y * W;
    for (int i = threadIdx.x; i < len; i += blockDim.x) sd[i] = drow[xa + i];
    for (int i = threadIdx.x; i < xe - xs; i += blockDim.x) sarm[i] = aref[xs + i];
    __syncthreads();

    // ---- A: votes and local prefix of this warp's segment (lane = d)
    const int d = a.d0 + 32 * g + lane;
    const int sa = warp * kHSeg, sb = min(len, sa + kHSeg);   // relative to xa
    static_assert(kHSeg <= 255, "k_hvote: local prefixes in one byte");
    uint32_t run = 0;
#pragma unroll 8
    for (int x = sa; x < sb; x++) {
        run += sd[x] == d ? 1u : 0u;
        P[x * 32 + lane] = (uint8_t)run;
    }
    T[warp * 32 + lane] = run;
    __syncthreads();
    // B: exclusive prefix of the segment totals (segment offsets), then C
    uint32_t offs = 0;
    for (int w = 0; w < warp; w++) offs += T[w * 32 + lane];
    __syncthreads();
    T[warp * 32 + lane] = offs;
    __syncthreads();
    hvote_out_quads<kHSegLog>(P, T, sarm, xe - xs, xs - xa, a.sh + ((size_t)y * W + xs) * a.dstride + g * 32,
                              a.dstride);
}

// ------------------------------------------------------------------ k_vagg
// Block = one column x of one reference view, a chunk of output rows.  The
// prefix range [ya, yb) is split into warp segments of 32 rows.  For each
// group of 32 disparities of the pass:
//   0. every warp moves its 32 slice rows (128 bytes each: the group's
//      disparities of one pixel) into Q[y - ya] with one TMA tile copy
//      (completing on the warp's mbarrier);
//   A. lane = disparity: the warp's 32 tile rows into registers, the
//      segment sum exchanged with the other warps, then the column prefix
//      (with its segment offset) written back in place (the rows of a
//      partial tile past the range are summed after the range's last row,
//      and the last warp's total is read by no other warp);
//   C. lane = output row: V(d) = Q(y + dn, d) - Q(y - up - 1, d) for the 32
//      disparities (Eq. 2: the sum over the vertical arm of the horizontal
//      sums; N does not depend on d, so the WTA compares V), running minimum
//      with the smallest d on ties (Eq. 3) in registers across groups; four
//      disparities per 16-byte shared load.
// Finally the running best is merged with earlier passes and written.
// Q rows are 36 words (144 bytes: the tile box is 32 disparities plus 4
// zero-filled words, a multiple of 16 bytes); in phase C the 16-byte loads
// of 32 rows spread over the 8 bank quads.
constexpr int kQS = 36;   // Q row stride in words
constexpr int kVSeg = 32; // rows per warp
constexpr int kQ0 = 64;   // Q[0] at word 64 (256 bytes): every warp's tile starts on a 128-byte boundary
constexpr uint32_t kVTileBytes = kVSeg * kQS * 4;

// words before the mbarriers: Q[-1] (zeros, at kQ0 - kQS) and Q [nw*32 rows:
// every warp's tile is 32 rows], T [nw][32], NQ [len], NT [nw]
__host__ __device__ inline size_t vagg_bar_word(int len, int nw)
{
    return ((size_t)kQ0 + (size_t)nw * kVSeg * kQS + nw * 32 + len + nw + 1) / 2 * 2;
}
__host__ __device__ inline size_t vagg_smem_words(int len, int nw) { return vagg_bar_word(len, nw) + 2 * nw; }

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *tm, int c0, int c1, int c2, uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
                 : "memory");
}
// TMA tile copy of the box at coordinates (c0, c1, c2, c3) of map `tm` to
// shared address `dst` (128-byte aligned), completing on mbarrier `bar`
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *tm, int c0, int c1, int c2, int c3,
                                            uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
                 : "memory");
}

// kMax: the WTA takes the largest V (the vote counts of Eq. 4) instead of the
// smallest: V is complemented, so the strict < keeps the smallest d on ties
// and the key merge across passes is unchanged
//
// kRow: the other aggregation order (the region is the union over q on p's
// horizontal arm of q's vertical segment): the block is one row y, the scan
// runs along x over the vertical segment sums, the window is p's horizontal
// arm and the region size adds u + d + 1 of every column.  Below, "rows" are
// the scan positions.
template <bool kMax, bool kRow>
__device__ __forceinline__ void vagg_body(const VArgs &a, int bx, int by, int bz)
{
    extern __shared__ __align__(16) uint32_t vsmem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int W = a.W, H = a.H, L1 = a.L1;
    const int fix = bx, view = by;              // the column x (kRow: the row y)
    const int E = kRow ? W : H;                 // extent of the scan
    const int ys = bz * a.chunk, ye = min(E, ys + a.chunk);
    const int ya = max(0, ys - L1), yb = min(E, ye + L1);
    const int len = yb - ya;
    auto pix = [&](int sp) -> size_t { return kRow ? (size_t)fix * W + sp : (size_t)sp * W + fix; };
    uint32_t *Q = vsmem + kQ0;                // [nw * 32][kQS], Q[-1] = 0
    uint32_t *T = Q + nw * kVSeg * kQS;       // [nw][32] segment sums
    uint32_t *NQ = T + nw * 32;               // [len] prefix of l + r + 1
    uint32_t *NT = NQ + len;                  // [nw]
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(vsmem) + 4u * (uint32_t)vagg_bar_word(len, nw) + 8u * warp;
    if (((uint32_t)__cvta_generic_to_shared(Q) & 127u) != 0) {   // the tile copies need 128-byte alignment
        if (threadIdx.x == 0 && a.status) atomicOr(a.status, kStatusAlign);
        return;
    }

    const CUtensorMap *tm = view ? &a.tm[1] : &a.tm[0];
    const uint32_t *arms = reinterpret_cast<const uint32_t *>(view ? a.arms[1] : a.arms[0]) + pix(0);
    const size_t astride = kRow ? 1 : (size_t)W;
    const int sa = warp * kVSeg, sb = min(len, sa + kVSeg);   // relative to ya
    const int nrow = max(0, sb - sa);
    const int ng = (a.dc + 31) / 32;
    const bool want_vol = a.vol != nullptr && view == a.vol_view;

    if (lane == 0) mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    __syncwarp();
    // group g's 32 rows of this warp's segment -> Q[sa .. sa + 31] (rows
    // past the image are zero-filled, rows past yb are read and unused; the
    // generic accesses of the previous group are ordered before the copy by
    // the block barrier and the proxy fence)
    auto issue = [&](int g) {
        if (nrow == 0 || lane != 0) return;
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mbar_expect_tx(bar, kVTileBytes);
        if (a.skip_copy) return;   // failure test: the barrier's phase never completes
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(Q + sa * kQS);
        if (a.tm_rank == 4)
            tma_load_4d(dst, tm, 0, g, kRow ? ya + sa : fix, kRow ? fix : ya + sa, bar);
        else
            tma_load_3d(dst, tm, 32 * g, kRow ? ya + sa : fix, kRow ? fix : ya + sa, bar);
    };
    issue(0);   // the first group's rows are in flight during the arm-word work

    // arm word of this lane's row and the region-size prefix (d independent)
    const int r = sa + lane;
    const bool rin = r < sb;
    const uint32_t aw = rin ? __ldg(arms + (size_t)(ya + r) * astride) : 0u;
    // window arms along the scan (computed where used: short live ranges),
    // and the segment length across it
    auto back = [&]() { return kRow ? (int)(aw & 0xffu) : (int)((aw >> 16) & 0xffu); };
    auto fwd = [&]() { return kRow ? (int)((aw >> 8) & 0xffu) : (int)(aw >> 24); };
    {
        uint32_t nv = !rin ? 0u : kRow ? ((aw >> 16) & 0xffu) + (aw >> 24) + 1u : (aw & 0xffu) + ((aw >> 8) & 0xffu) + 1u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {   // inclusive scan across the segment's rows
            const uint32_t t = __shfl_up_sync(0xffffffffu, nv, o);
            if (lane >= o) nv += t;
        }
        if (rin) NQ[r] = nv;
        if (lane == 31) NT[warp] = nv;
    }
    const bool out_row = rin && ya + r >= ys && ya + r < ye;
    uint32_t bv = 0xffffffffu, bd = 0;
    if (warp == 0) Q[-kQS + lane] = 0u;   // Q[-1]: read by rows whose up arm reaches the top
    for (int g = 0; g < ng; g++) {
        // ---- A: this warp's rows of the slice column, lane = disparity
        const bool lost = nrow > 0 && !mbar_wait(bar, (uint32_t)(g & 1), a.wait_limit);
        if (__syncthreads_or(lost)) {
            // a copy did not complete: report it, issue no further copies,
            // and give this warp's copy a last bounded wait before the
            // block's shared memory is released
            if (lost) {
                if (lane == 0 && a.status) atomicOr(a.status, kStatusCopyTimeout);
                mbar_wait(bar, (uint32_t)(g & 1), a.wait_limit);
            }
            return;
        }
        uint32_t *q = Q + sa * kQS + lane;
        uint32_t tot = 0;
        uint32_t v[kVSeg];
#pragma unroll
        for (int u = 0; u < kVSeg; u++) { v[u] = q[u * kQS]; tot += v[u]; }
        T[warp * 32 + lane] = tot;
        __syncthreads();
        uint32_t run = 0;
        for (int w = 0; w < warp; w++) run += T[w * 32 + lane];
        if (g == 0) {
            // region-size offsets (once)
            uint32_t noff = 0;
            for (int w = 0; w < warp; w++) noff += NT[w];
            if (rin) NQ[r] += noff;
        }
#pragma unroll
        for (int u = 0; u < kVSeg; u++) {
            run += v[u];
            q[u * kQS] = run;
        }
        __syncthreads();
        // ---- C: lane = output row, loop over the group's disparities
        const int dbase = a.d0 + g * 32;
        const int nlive = max(0, min(32, min(a.dc - g * 32, a.D - dbase)));
        if (out_row) {
            const uint32_t *qh = Q + (r + fwd()) * kQS;
            const int lo = r - back() - 1;           // >= -1
            const uint32_t *ql = Q + lo * kQS;
            // running minimum; strict < keeps the smallest d on ties
            uint32_t bj = 0xffffffffu, bmin = bv;
            if (nlive == 32) {
                const uint4 *qh4 = reinterpret_cast<const uint4 *>(qh), *ql4 = reinterpret_cast<const uint4 *>(ql);
#pragma unroll 2
                for (int j4 = 0; j4 < 8; j4++) {
                    const uint4 h4 = qh4[j4], l4 = ql4[j4];
                    const uint32_t hv[4] = {h4.x, h4.y, h4.z, h4.w}, lv[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        const uint32_t vv = kMax ? ~(hv[k] - lv[k]) : hv[k] - lv[k];
                        bj = vv < bmin ? (uint32_t)(4 * j4 + k) : bj;
                        bmin = min(bmin, vv);
                    }
                }
            } else {
                for (int j = 0; j < nlive; j++) {
                    const uint32_t vv = kMax ? ~(qh[j] - ql[j]) : qh[j] - ql[j];
                    bj = vv < bmin ? (uint32_t)j : bj;
                    bmin = min(bmin, vv);
                }
            }
            if (bj != 0xffffffffu) { bv = bmin; bd = (uint32_t)dbase + bj; }
            if (want_vol) {
                const uint32_t n = NQ[r + fwd()] - (lo >= 0 ? NQ[lo] : 0u);
                for (int j = 0; j < nlive; j++) {
                    const uint32_t vv = qh[j] - ql[j];
                    a.vol[(size_t)(dbase - a.dmin + j) * H * W + pix(ya + r)] = float(vv) / (float(n) * a.S);
                }
            }
        }
        __syncthreads();   // Q and T are reused by the next group
        if (g + 1 < ng) issue(g + 1);
    }
    // ---- merge with earlier passes, write the disparity (last pass) or state
    if (!out_row) return;
    unsigned long long *best = view ? a.best[1] : a.best[0];
    int16_t *disp = view ? a.disp[1] : a.disp[0];
    float *cost = view ? a.cost[1] : a.cost[0];
    const size_t i = pix(ya + r);
    unsigned long long key = ((unsigned long long)bv << 32) | bd;
    if (!a.first) {
        const unsigned long long prev = best[i];
        key = prev <= key ? prev : key;   // earlier passes hold smaller d
    }
    if (a.last) {
        const bool invalid = kMax && (a.mask[i] < a.dmin || a.mask[i] >= a.D);   // Eq. 4: no vote, stays invalid
        disp[i] = invalid ? (int16_t)-1 : (int16_t)(key & 0xffffffffu);
        if (cost) {
            const int lo = r - back() - 1;
            const uint32_t n = NQ[r + fwd()] - (lo >= 0 ? NQ[lo] : 0u);
            cost[i] = float(uint32_t(key >> 32)) / (float(n) * a.S);
        }
    } else {
        best[i] = key;
    }
}

// ------------------------------------------------------------------ k_lr
__device__ __forceinline__ void lr_body(const LrArgs &a, size_t i)
{
    if (i >= (size_t)a.W * a.H) return;
    const int x = int(i % a.W);
    const int d = a.dl[i];
    int16_t r = -1;
    if (a.tol < 0) r = (int16_t)d;
    else if (d >= 0 && x - d >= 0) {
        const int d2 = a.dr[i - d];
        if (d2 >= 0 && abs(d - d2) <= a.tol) r = (int16_t)d;
    }
    a.out[i] = r;
}

// ------------------------------------------------------ quarter size, depth
// Sect. 4: the pair is matched at half of each axis; channel c of output
// pixel (x, y) is the rounded mean (sum + 2) >> 2 of its 2x2 input block.
__global__ void __launch_bounds__(256) k_down(const DownArgs a)
{
    pdl_enter();
    const int Wh = a.W / 2, Hh = a.H / 2;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= Wh || y >= Hh) return;
    const uint8_t *s0 = a.src[blockIdx.z] + ((size_t)(2 * y) * a.W + 2 * x) * 3;
    const uint8_t *s1 = s0 + (size_t)a.W * 3;
    uint8_t *d = a.dst[blockIdx.z] + ((size_t)y * Wh + x) * 3;
#pragma unroll
    for (int c = 0; c < 3; c++) d[c] = (uint8_t)((s0[c] + s0[3 + c] + s1[c] + s1[3 + c] + 2) >> 2);
}

// Sect. 4.4: the half-size disparity doubled back to full size, Z = f B / (2 d)
// on the 2x2 block of each half-size pixel; 0 (missing, Eq. 14) where d <= 0
// and on an odd last row or column.  Thread = one 2x2 block (hx, hy) of the
// ceil(W/2) x ceil(H/2) blocks.
__global__ void __launch_bounds__(256) k_depth(const DepthArgs a)
{
    pdl_enter();
    const int hx = blockIdx.x * blockDim.x + threadIdx.x, hy = blockIdx.y;
    if (2 * hx >= a.W) return;
    const int Wh = a.W / 2;
    float z = 0.0f;
    if (hx < Wh && hy < a.H / 2) {
        const int d = a.disp[(size_t)hy * Wh + hx];
        if (d > 0) z = a.fb / (2.0f * (float)d);
    }
    const int x = 2 * hx;
    for (int y = 2 * hy; y < min(a.H, 2 * hy + 2); y++) {
        float *o = a.out + (size_t)y * a.W + x;
        o[0] = z;
        if (x + 1 < a.W) o[1] = z;
    }
}

// ------------------------------------------------------------------ batches
// Every stage is one launch over all pairs of a batch (a single pair is a
// batch of one).  The pairs' arguments travel in the kernel parameters; the
// flat block index is mapped to (pair, block of that pair's own grid).
template <class A, int N>
struct Batch {
    int n;
    int off[N + 1];   // first flat block of each pair; off[n] = total
    int gx[N], gy[N]; // the pair's own grid is gx x gy x gz
    A p[N];
};

// launch with programmatic stream serialization (the kernel calls pdl_enter
// before any global memory access)
template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <class A, int N>
__device__ __forceinline__ int batch_pair(const Batch<A, N> &b, int flat, int &bx, int &by, int &bz)
{
    int lo = 0, hi = b.n - 1;
    while (lo < hi) {   // last pair with off <= flat
        const int mid = (lo + hi + 1) >> 1;
        if (b.off[mid] <= flat) lo = mid;
        else hi = mid - 1;
    }
    const int local = flat - b.off[lo];
    bx = local % b.gx[lo];
    const int t = local / b.gx[lo];
    by = t % b.gy[lo];
    bz = t / b.gy[lo];
    return lo;
}

template <int N, bool kMax>
__global__ void __launch_bounds__(256) k_smooth(const __grid_constant__ Batch<SmoothArgs, N> b)
{
    pdl_enter();
    int bx, by, bz;
    const int i = batch_pair(b, blockIdx.x, bx, by, bz);
    smooth_body<kMax>(b.p[i], bx * 256 + threadIdx.x, by);
}

// kRows 0: the flat mapping (images in device memory); else blocks of
// kRows rows per thread (images in host memory)
template <int N, int kRows = 0>
__global__ void __launch_bounds__(256) k_pack(const __grid_constant__ Batch<PackArgs, N> b)
{
    pdl_enter();
    int bx, by, bz;
    const int i = batch_pair(b, blockIdx.x, bx, by, bz);
    if (kRows == 0) pack_body(b.p[i], bx * 256 + threadIdx.x, by);
    else pack_rows_body<kRows ? kRows : 1>(b.p[i], bx * 256 + threadIdx.x, by);
}

template <int CW, int CH, int N>
__global__ void __launch_bounds__(kTX * kTY) k_prep(const __grid_constant__ Batch<PrepArgs, N> b)
{
    pdl_enter();
    int bx, by, bz;
    const int i = batch_pair(b, blockIdx.x, bx, by, bz);
    prep_body<CW, CH>(b.p[i], bx, by, bz);
}

// kWide: blocks of more than kHNarrow warps (rows wider than 640 columns)
template <int N, bool kWide>
__global__ void __launch_bounds__(kWide ? 1024 : kHNarrow * 32) k_hagg(const __grid_constant__ Batch<HArgs, N> b)
{
    pdl_enter();
    int bx, by, bz;
    const int i = batch_pair(b, blockIdx.x, bx, by, bz);
    hagg_body(b.p[i], bx, by, bz);
}

template <int N, bool kMax, bool kRow = false>
__global__ void __launch_bounds__(16 * 32, 2) k_vagg(const __grid_constant__ Batch<VArgs, N> b)
{
    pdl_enter();
    int bx, by, bz;
    const int i = batch_pair(b, blockIdx.x, bx, by, bz);
    vagg_body<kMax, kRow>(b.p[i], bx, by, bz);
}

template <int N>
__global__ void __launch_bounds__(1024) k_vcost(const __grid_constant__ Batch<HArgs, N> b)
{
    pdl_enter();
    int bx, by, bz;
    const int i = batch_pair(b, blockIdx.x, bx, by, bz);
    vcost_body(b.p[i], bx, by, bz);
}

template <int N>
__global__ void __launch_bounds__(16 * 32) k_hvote(const __grid_constant__ Batch<HVArgs, N> b)
{
    pdl_enter();
    int bx, by, bz;
    const int i = batch_pair(b, blockIdx.x, bx, by, bz);
    hvote_body(b.p[i], bx, by, bz);
}

template <int N>
__global__ void __launch_bounds__(256) k_lr(const __grid_constant__ Batch<LrArgs, N> b)
{
    pdl_enter();
    int bx, by, bz;
    const int i = batch_pair(b, blockIdx.x, bx, by, bz);
    lr_body(b.p[i], (size_t)bx * 256 + threadIdx.x);
}

__global__ void k_extract_census(const uint4 *__restrict__ rec, int W, int H, int rpitch,
                                 unsigned long long *out)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)W * H) return;
    const uint4 r = rec[(i / W) * rpitch + i % W];
    out[i] = ((unsigned long long)r.y << 32) | r.x;
}

} // namespace dco

// ====================================================================== host
using namespace dco;

namespace {

struct ProfEvent {
    const char *name;
    cudaEvent_t a, b;
};

struct ProfAgg {
    std::string name;
    int launches = 0;
    double ms = 0.0;
};

struct Derived {
    int L1;
    uint32_t Sint;
    float S;
    int order;   // aggregation order: 0 horizontal then vertical, 1 vertical then horizontal
    int dmin;    // smallest disparity of the search
    int hchunk, vchunk;   // tile shapes of the two 1-D passes (0: automatic)
};

struct Layout {
    size_t rgbx[2], grey[2], rec[2], cen[2], col[2], arms[2], atmp[2], best[2], disp[2], sh[2], vtmp, total;
    int dc, dstride, npass, rpitch, phw;
};

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

bool derive(const dco_params &p, Derived &d)
{
    d.L1 = p.arm_l1;
    // fixed-point scale: the largest region, (2*L1+1)^2 costs of at most 1
    // (+1 unit of rounding each), must stay below 2^32
    const double n = double(2 * p.arm_l1 + 1) * double(2 * p.arm_l1 + 1);
    double s = std::floor(4294967295.0 / n) - 1.0;
    s = std::min(s, 1048576.0);
    d.Sint = (uint32_t)s;
    d.S = (float)s;
    d.order = p.agg_order;
    d.dmin = p.d_min;
    d.hchunk = p.h_chunk;
    d.vchunk = p.v_chunk;
    return true;
}

// a tile shape: 0 (automatic) or 32 .. 16384 positions
bool tile_valid(int c) { return c == 0 || (c >= 32 && c <= 16384); }

bool params_valid(const dco_params &p)
{
    if (!(p.lambda_ad > 0.f) || !(p.lambda_census > 0.f) || !(p.eps > 0.f) || !(p.gamma_l >= 0.f))
        return false;
    if (p.census_w < 1 || p.census_h < 1 || !(p.census_w & 1) || !(p.census_h & 1)) return false;
    if (p.census_w > kMaxCW || p.census_h > kMaxCH || p.census_w * p.census_h - 1 > 64) return false;
    if (p.arm_l1 < 1 || p.arm_l1 > kMaxL1 || p.arm_l2 < 0 || p.tau1 < 0 || p.tau2 < 0) return false;
    if (p.d_chunk < 0) return false;
    if (p.vote_iters < 0 || p.vote_iters > 64) return false;
    if (p.smooth_arms != 0 && p.smooth_arms != 1) return false;
    if (p.agg_order != 0 && p.agg_order != 1) return false;
    if (p.d_min < 0 || p.d_min > 255) return false;
    if (!tile_valid(p.h_chunk) || !tile_valid(p.v_chunk)) return false;
    return true;
}

bool dims_valid(int W, int H, int D, int dmin = 0)
{
    return W >= 1 && H >= 1 && W <= 16384 && H <= 16384 && D >= 1 && dmin >= 0 && dmin + D <= 256 && dmin + D <= W;
}

Layout make_layout(int W, int H, int D, const dco_params &p, int dc_override = 0)
{
    Layout L{};
    const size_t npx = (size_t)W * H;
    int dc = dc_override > 0 ? dc_override : p.d_chunk;
    if (dc <= 0) {
        // automatic: slices of both views within ~96 MB so the producer and
        // consumer of a pass meet in L2; at least one warp of disparities
        const size_t cap = 96u << 20;
        int full = (D + 31) / 32 * 32;
        if (8 * npx * (size_t)full <= cap) dc = D;
        else {
            size_t fit = cap / (8 * npx);
            dc = (int)std::max<size_t>(32, fit / 32 * 32);
        }
    }
    dc = std::min(dc, D);
    L.dc = dc;
    L.dstride = (dc + 31) / 32 * 32;
    L.npass = (D + dc - 1) / dc;
    size_t off = 0;
    L.rpitch = W + 2 * kRPad;
    L.phw = ((W + 1) / 2 + 3) / 4 * 4;
    for (int v = 0; v < 2; v++) { L.rgbx[v] = off; off = align_up(off + 4 * npx); }
    for (int v = 0; v < 2; v++) { L.grey[v] = off; off = align_up(off + npx); }
    for (int v = 0; v < 2; v++) { L.rec[v] = off; off = align_up(off + 16 * (size_t)H * L.rpitch); }
    // candidate planes, 16 bytes of slack each (the bulk copies end on 16-byte boundaries)
    for (int v = 0; v < 2; v++) { L.cen[v] = off; off = align_up(off + 8 * (size_t)H * 2 * L.phw + 16); }
    for (int v = 0; v < 2; v++) { L.col[v] = off; off = align_up(off + 4 * (size_t)H * 2 * L.phw + 16); }
    // arms: 16 bytes of slack, read by the cost pass's bulk copies past the last pixel
    for (int v = 0; v < 2; v++) { L.arms[v] = off; off = align_up(off + 4 * npx + 16); }
    for (int v = 0; v < 2; v++) { L.atmp[v] = off; off = align_up(off + (p.smooth_arms ? 4 * npx : 0)); }
    for (int v = 0; v < 2; v++) { L.best[v] = off; off = align_up(off + (L.npass > 1 ? 8 * npx : 0)); }
    for (int v = 0; v < 2; v++) { L.disp[v] = off; off = align_up(off + 2 * npx); }
    for (int v = 0; v < 2; v++) { L.sh[v] = off; off = align_up(off + 4 * npx * (size_t)L.dstride); }
    L.vtmp = off;   // second map of the Eq. 4 rounds
    off = align_up(off + (p.vote_iters > 0 ? 2 * npx : 0));
    L.total = off;
    return L;
}

// H geometry: one block per (row, chunk of output columns, view, group);
// the block's prefix range is the chunk plus an L1 reach on both sides
struct HGeom {
    int chunk, nw;
    size_t smem;
    dim3 grid;
};

// Output positions per block of a first-pass line of n positions: the whole
// line up to kHMaxLen, else 512 (want = 0); otherwise `want`, capped so that
// a block's prefix range (chunk + 2 L1 halo) stays within kHMaxLen.
int first_pass_chunk(int n, int L1, int want)
{
    if (want <= 0) return n <= kHMaxLen ? n : 512;
    int c = std::min(want, n);
    if (c < n || n > kHMaxLen) c = std::min(c, kHMaxLen - 2 * L1);
    return c;
}

// the other aggregation order: k_vcost walks columns (one chunk of rows per
// block while it fits 32 warps of 32 rows), k_vagg<.., kRow> rows (the scan
// range along x at most 512 columns, like k_vagg's rows)
HGeom vcost_geom(int W, int H, int dc, int L1, int want)
{
    HGeom g{};
    g.chunk = first_pass_chunk(H, L1, want);
    const int len = std::min(H, g.chunk + 2 * L1);
    g.nw = (len + kHSegCost - 1) / kHSegCost;
    g.smem = CSmem(len, g.chunk, g.nw).total;
    g.grid = dim3(W, (H + g.chunk - 1) / g.chunk, 2 * ((dc + 31) / 32));
    return g;
}

HGeom hagg_geom(int W, int H, int dc, int L1, int want)
{
    HGeom g{};
    g.chunk = first_pass_chunk(W, L1, want);
    const int len = std::min(W, g.chunk + 2 * L1);
    g.nw = (len + kHSegCost - 1) / kHSegCost;
    g.smem = HSmem(len, g.chunk, g.nw).total;
    const int ngroups = (dc + 31) / 32;
    g.grid = dim3((W + g.chunk - 1) / g.chunk, H, 2 * ngroups);
    return g;
}

// V geometry: one block per (column, view, chunk of output rows)
struct VGeom {
    int chunk, nw, seglog;
    size_t smem;
    dim3 grid;
};

VGeom vagg_geom(int W, int H, int L1, int want)
{
    VGeom g{};
    // at most 16 warps of 32 rows: the prefix range (chunk + 2*L1) <= 512;
    // balanced chunks of at most `want` rows (automatic: whole columns up
    // to 512 rows, else at most 512 - 2 kMaxL1)
    int nchunks;
    if (want <= 0) {
        nchunks = H <= 512 ? 1 : (H + (512 - 2 * kMaxL1) - 1) / (512 - 2 * kMaxL1);
    } else {
        int c = std::min(want, H);
        if (c < H || H > 512) c = std::min(c, 512 - 2 * L1);
        nchunks = (H + c - 1) / c;
    }
    g.chunk = (H + nchunks - 1) / nchunks;
    const int len = std::min(H, g.chunk + 2 * L1);
    g.seglog = 5;   // 32 rows per warp, one output row per lane
    g.nw = (len + kVSeg - 1) / kVSeg;
    g.smem = vagg_smem_words(len, g.nw) * 4;
    g.grid = dim3(W, 2, nchunks);
    return g;
}

// ---- TMA tile maps of the slices (k_vagg)
using TmapEncode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

TmapEncode tmap_encoder()
{
    static TmapEncode fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<TmapEncode>(f);
    });
    return fn;
}


} // namespace

struct dco_stereo {
    int device = 0;
    size_t budget = 0;
    char *ws = nullptr;
    size_t ws_cap = 0;
    int *d_status = nullptr;
    float *d_tables = nullptr;
    float *h_tables = nullptr;   // pinned staging of the tables
    bool tab_valid = false;
    float tab_key[4] = {0, 0, 0, 0};
    int tab_l1 = -1;
    uint8_t *stage = nullptr;
    size_t stage_cap = 0;
    bool profiling = false;
    int test_flags = 0;                      // DCO_TEST_* failure tests (0 in normal use)
    int groups_last = 1;                     // admission groups of the last batch call
    unsigned long long launches = 0;
    std::vector<ProfEvent> pending;
    std::vector<cudaEvent_t> pool;
    std::vector<ProfAgg> agg;
    std::string last_error;
    int *dn_pin = nullptr;                   // pinned convergence flag of the densify solve
    cudaEvent_t dn_ev[2] = {nullptr, nullptr};
    cudaStream_t dn_stream = nullptr;        // private stream the iteration batch is captured on
    cudaGraphExec_t dn_exec = nullptr;       // one captured batch of iterations
    std::vector<unsigned char> dn_key;       // the arguments it was captured with
    int dn_iters = 0;
    double dn_relres = 0.0;
};

namespace {

// A failed runtime call also leaves its error as the thread's last error;
// it is reported here and then dropped, so that the launch checks of the
// next call (cudaGetLastError after a launch) see only their own launches.
dco_status cuda_fail(dco_stereo *h, cudaError_t e, const char *what)
{
    if (h) h->last_error = std::string(what) + ": " + cudaGetErrorString(e);
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? DCO_ENOMEM : DCO_ECUDA;
}

// Entry of a call that launches work: h's device made current, and a
// non-sticky error that an earlier runtime call left in this thread dropped
// (it belongs to that call, not to this one's launches).
cudaError_t enter_device(const dco_stereo *h)
{
    const cudaError_t e = cudaSetDevice(h->device);
    (void)cudaGetLastError();
    return e;
}

// status word -> call status: a lost tile copy is a timed-out wait, any
// other bit a failed internal check
dco_status status_of_word(int v)
{
    if (v == 0) return DCO_OK;
    return (v & kStatusCopyTimeout) ? DCO_ETIMEOUT : DCO_EDEVICE;
}

#define DCO_CUDA(h, call)                                              \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);       \
    } while (0)

cudaEvent_t take_event(dco_stereo *h)
{
    if (!h->pool.empty()) {
        cudaEvent_t e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void collect_profile(dco_stereo *h)
{
    for (auto &pe : h->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pe.a, pe.b) == cudaSuccess) {
            ProfAgg *slot = nullptr;
            for (auto &g : h->agg)
                if (g.name == pe.name) slot = &g;
            if (!slot) {
                h->agg.push_back(ProfAgg{pe.name, 0, 0.0});
                slot = &h->agg.back();
            }
            slot->launches += 1;
            slot->ms += ms;
        }
        h->pool.push_back(pe.a);
        h->pool.push_back(pe.b);
    }
    h->pending.clear();
}

struct ProfScope {
    dco_stereo *h;
    cudaStream_t s;
    ProfEvent ev{};
    // name == nullptr: a launch being captured into a graph (counted when the
    // graph runs, never timed)
    ProfScope(dco_stereo *h_, cudaStream_t s_, const char *name) : h(name ? h_ : nullptr), s(s_)
    {
        if (!h) return;
        h->launches++;
        if (h->profiling) {
            ev.name = name;
            ev.a = take_event(h);
            ev.b = take_event(h);
            cudaEventRecord(ev.a, s);
        }
    }
    ~ProfScope()
    {
        if (h && h->profiling) {
            cudaEventRecord(ev.b, s);
            h->pending.push_back(ev);
        }
    }
};

dco_status ensure_ws(dco_stereo *h, size_t need)
{
    if (need <= h->ws_cap) return DCO_OK;
    if (h->budget && need > h->budget) {
        h->last_error = "workspace of " + std::to_string(need) + " bytes exceeds the budget of " +
                        std::to_string(h->budget);
        return DCO_EBUDGET;
    }
    if (h->ws) {
        DCO_CUDA(h, cudaDeviceSynchronize());
        cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_cap = 0;
    }
    DCO_CUDA(h, cudaMalloc((void **)&h->ws, need));
    h->ws_cap = need;
    return DCO_OK;
}

// Eq. 1 tables, evaluated in double on the host and rounded once to float:
//   [0, kTabAD)   1 - exp(-(k/3) / lambda_AD), k = 0..765 (the channel sum);
//   [kTabAD, +kTabCen)   1 - exp(-h / lambda_census), h = 0..64;
//   [kTabAD + kTabCen, +kTabAlpha)   alpha(Lmin) * S.
void fill_tables(float *t, const dco_params &p, const Derived &dv)
{
    for (int k = 0; k < kTabAD; k++)
        t[k] = k <= 765 ? (float)(1.0 - std::exp(-(k / 3.0) / (double)p.lambda_ad)) : 1.0f;
    for (int k = 0; k < kTabCen; k++)
        t[kTabAD + k] = k <= 64 ? (float)(1.0 - std::exp(-(double)k / (double)p.lambda_census)) : 1.0f;
    for (int l = 0; l < kTabAlpha; l++) {
        const double alpha = 1.0 - std::exp(-(double)p.gamma_l / ((double)l + (double)p.eps));
        t[kTabAD + kTabCen + l] = (float)(alpha * (double)dv.Sint);
    }
}

dco_status ensure_tables(dco_stereo *h, const dco_params &p, const Derived &dv, cudaStream_t s)
{
    const float key[4] = {p.lambda_ad, p.lambda_census, p.gamma_l, p.eps};
    if (h->tab_valid && !std::memcmp(key, h->tab_key, sizeof key) && h->tab_l1 == p.arm_l1) return DCO_OK;
    float *t = h->h_tables;
    fill_tables(t, p, dv);
    DCO_CUDA(h, cudaMemcpyAsync(h->d_tables, t, sizeof(float) * kTabFloats, cudaMemcpyHostToDevice, s));
    // the pinned staging buffer is reused by the next upload: wait for this one
    DCO_CUDA(h, cudaStreamSynchronize(s));
    std::memcpy(h->tab_key, key, sizeof key);
    h->tab_l1 = p.arm_l1;
    h->tab_valid = true;
    return DCO_OK;
}

template <class T>
T *ws_ptr(dco_stereo *h, size_t off) { return reinterpret_cast<T *>(h->ws + off); }


// grey/colour packing and census + arms for nimg images (1 or 2); arms of
// image 0 go to arms0 (the caller's buffer for the arms entry point)
// ----------------------------------------------------------- batched launches
constexpr int kBatchMax = 64;   // pairs per launch (kernel parameter space)
// pairs per launch of a kind of argument block: the V blocks carry two
// tensor maps, so half as many fit the 32764 bytes of kernel parameters
template <class A> constexpr int batch_max() { return sizeof(A) > 256 ? kBatchMax / 2 : kBatchMax; }
static_assert(sizeof(Batch<VArgs, batch_max<VArgs>()>) <= 32764, "kernel parameters of a full V batch");
static_assert(sizeof(Batch<HArgs, batch_max<HArgs>()>) <= 32764, "kernel parameters of a full H batch");
constexpr int kVBatch = batch_max<VArgs>();

// The dynamic shared-memory limit is an attribute of the kernel on a device,
// shared by every handle and thread of the process: it is raised under a lock
// and never lowered, so a warmed-up process makes no attribute calls (safe
// inside stream capture) and no handle can shrink another's limit.
std::mutex g_smem_mu;
std::map<std::pair<int, const void *>, size_t> g_smem_set;

dco_status opt_in_smem(dco_stereo *h, const void *kernel, size_t smem)
{
    std::lock_guard<std::mutex> lock(g_smem_mu);
    size_t &done = g_smem_set[{h->device, kernel}];
    if (smem <= done) return DCO_OK;
    DCO_CUDA(h, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    done = smem;
    return DCO_OK;
}

template <class A>
struct Item {
    A a;
    int gx, gy, gz;   // the pair's own grid
};

template <class A, int N, class K>
dco_status launch_group(dco_stereo *h, cudaStream_t s, const char *name, K kernel, const Item<A> *it, int n,
                        int block, size_t smem)
{
    Batch<A, N> b;
    std::memset(&b, 0, sizeof b);
    b.n = n;
    b.off[0] = 0;
    for (int i = 0; i < n; i++) {
        b.gx[i] = it[i].gx;
        b.gy[i] = it[i].gy;
        b.p[i] = it[i].a;
        b.off[i + 1] = b.off[i] + it[i].gx * it[i].gy * it[i].gz;
    }
    if (b.off[n] == 0) return DCO_OK;
    if (smem > (48u << 10)) {
        dco_status st = opt_in_smem(h, reinterpret_cast<const void *>(kernel), smem);
        if (st != DCO_OK) return st;
    }
    ProfScope ps(h, s, name);
    cudaError_t e = launch_pdl(kernel, dim3((unsigned)b.off[n]), dim3((unsigned)block), smem, s, b);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        h->last_error = std::string(name) + " launch (" + std::to_string(n) + " pairs, " + std::to_string(b.off[n]) +
                        " blocks of " + std::to_string(block) + " threads, " + std::to_string(smem) +
                        " B shared): " + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? DCO_ENOMEM : DCO_ECUDA;
    }
    return DCO_OK;
}

// one launch for a single pair (small parameter block), else groups of
// batch_max<A>() (kn is the kernel instance for that many)
template <class A, class K1, class KN>
dco_status launch_items(dco_stereo *h, cudaStream_t s, const char *name, K1 k1, KN kn,
                        const std::vector<Item<A>> &items, int block, size_t smem)
{
    constexpr int nmax = batch_max<A>();
    if (items.empty()) return DCO_OK;
    if (items.size() == 1) return launch_group<A, 1>(h, s, name, k1, items.data(), 1, block, smem);
    for (size_t i = 0; i < items.size(); i += nmax) {
        const int n = (int)std::min<size_t>(nmax, items.size() - i);
        dco_status st = launch_group<A, nmax>(h, s, name, kn, items.data() + i, n, block, smem);
        if (st != DCO_OK) return st;
    }
    return DCO_OK;
}

// one pair of a run
struct Job {
    const uint8_t *left = nullptr, *right = nullptr;
    int W = 0, H = 0, D = 0;
    int16_t *out = nullptr, *disp_l = nullptr, *disp_r = nullptr;
    float *cost_l = nullptr, *cost_r = nullptr, *vol = nullptr;
    int vol_view = 0;
    uchar4 *arms0 = nullptr;   // stage entry point: arms of image 0 go here
    int dchunk = 0;                  // this pair's pass width (0: the call's parameters)
    int hchunk = 0, vchunk = 0;      // this pair's tile shapes (0: the call's parameters)
    int host_in = -1;                // images in host memory: 1, in device memory: 0, -1: ask the driver
    const int16_t *vsrc = nullptr;   // Eq. 4 round: map voted on (null: no vote)
    int16_t *vdst = nullptr;         //   and the map written
    Layout L{};
    size_t base = 0;           // workspace offset of this pair
};

// workspace plan for all jobs; the pass width shrinks (same for all pairs)
// until the plan fits the handle's budget
dco_status plan_jobs(dco_stereo *h, const dco_params &p, std::vector<Job> &jobs, size_t &total)
{
    // a pair's own pass width (j.dchunk > 0) replaces the call's; a budget
    // override caps both
    auto plan = [&](int dc_override) {
        size_t t = 0;
        for (auto &j : jobs) {
            int dc = j.dchunk > 0 ? j.dchunk : 0;
            if (dc_override > 0) dc = dc > 0 ? std::min(dc, dc_override) : dc_override;
            j.L = make_layout(j.W, j.H, j.D, p, dc);
            j.base = t;
            t = align_up(t + j.L.total);
        }
        return t;
    };
    total = plan(0);
    if (h->budget && total > h->budget) {
        int widest = 32;
        for (auto &j : jobs) widest = std::max(widest, (j.L.dc + 31) / 32 * 32);
        for (int dc = widest; dc >= 32 && total > h->budget; dc -= 32) total = plan(dc);
    }
    return DCO_OK;
}

template <class T>
T *jptr(dco_stereo *h, const Job &j, size_t off) { return ws_ptr<T>(h, j.base + off); }

// grey/colour packing and census + arms for nimg images of every job
// images the kernels read from host memory (pinned or registered; over
// NVLink-C2C on Grace systems)
constexpr int kPackHostRows = 4;   // rows per k_pack thread for those
bool in_host_memory(const void *p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost;
}

dco_status launch_prep(dco_stereo *h, const dco_params &p, const Derived &dv, const std::vector<Job> &jobs,
                       int nimg, cudaStream_t s)
{
    std::vector<Item<PackArgs>> pk, pk_host;
    std::vector<Item<PrepArgs>> pr;
    for (const Job &j : jobs) {
        const int npx = j.W * j.H;
        Item<PackArgs> a{};
        a.a.rgb[0] = j.left; a.a.rgb[1] = j.right;
        for (int v = 0; v < 2; v++) {
            a.a.rgbx[v] = jptr<uint32_t>(h, j, j.L.rgbx[v]);
            a.a.grey[v] = jptr<uint8_t>(h, j, j.L.grey[v]);
        }
        a.a.npx = npx;
        a.a.W = j.W;
        a.a.k1 = 0x00100401u * (uint32_t)(std::min(p.tau1, 256) + 511);   // tau1 in every 10-bit field
        a.gy = nimg;
        a.gz = 1;
        if (j.host_in > 0 || (j.host_in < 0 && (in_host_memory(j.left) || in_host_memory(j.right)))) {
            a.gx = (((j.W + 3) / 4) * ((j.H + kPackHostRows - 1) / kPackHostRows) + 255) / 256;
            pk_host.push_back(a);
        } else {
            a.gx = (npx + 1023) / 1024;   // 256 threads x 4 pixels
            pk.push_back(a);
        }
        Item<PrepArgs> b{};
        for (int v = 0; v < 2; v++) {
            b.a.rgbx[v] = jptr<uint32_t>(h, j, j.L.rgbx[v]);
            b.a.grey[v] = jptr<uint8_t>(h, j, j.L.grey[v]);
            b.a.rec[v] = jptr<uint4>(h, j, j.L.rec[v]) + kRPad;
            b.a.cen[v] = jptr<uint2>(h, j, j.L.cen[v]);
            b.a.col[v] = jptr<uint32_t>(h, j, j.L.col[v]);
            b.a.arms[v] = jptr<uchar4>(h, j, j.L.arms[v]);
        }
        b.a.phw = j.L.phw;
        if (j.arms0) b.a.arms[0] = j.arms0;
        b.a.tables = h->d_tables;
        b.a.W = j.W; b.a.H = j.H; b.a.rpitch = j.L.rpitch;
        b.a.cw = p.census_w; b.a.ch = p.census_h;
        b.a.L1 = dv.L1; b.a.L2 = p.arm_l2; b.a.tau1 = p.tau1; b.a.tau2 = p.tau2;
        b.gx = (j.W + kTX - 1) / kTX;
        b.gy = (j.H + kTY - 1) / kTY;
        b.gz = nimg;
        pr.push_back(b);
    }
    dco_status st = launch_items(h, s, "k_pack", k_pack<1>, k_pack<kBatchMax>, pk, 256, 0);
    if (st != DCO_OK) return st;
    st = launch_items(h, s, "k_pack", k_pack<1, kPackHostRows>, k_pack<kBatchMax, kPackHostRows>, pk_host, 256, 0);
    if (st != DCO_OK) return st;
    if (p.census_w == 9 && p.census_h == 7)
        st = launch_items(h, s, "k_prep", k_prep<9, 7, 1>, k_prep<9, 7, kBatchMax>, pr, kTX * kTY, 0);
    else
        st = launch_items(h, s, "k_prep", k_prep<0, 0, 1>, k_prep<0, 0, kBatchMax>, pr, kTX * kTY, 0);
    if (st != DCO_OK || !p.smooth_arms) return st;
    // Sect. 4.1 smoothing: arms -> 3x3 minimum (atmp) -> 3x3 maximum (arms, records)
    std::vector<Item<SmoothArgs>> er, di;
    for (size_t k = 0; k < jobs.size(); k++) {
        const Job &j = jobs[k];
        Item<SmoothArgs> e{};
        for (int v = 0; v < 2; v++) {
            e.a.src[v] = pr[k].a.arms[v];
            e.a.dst[v] = jptr<uchar4>(h, j, j.L.atmp[v]);
        }
        e.a.tables = h->d_tables;
        e.a.W = j.W; e.a.H = j.H; e.a.rpitch = j.L.rpitch;
        e.gx = (j.W * j.H + 255) / 256; e.gy = nimg; e.gz = 1;
        er.push_back(e);
        Item<SmoothArgs> d = e;
        for (int v = 0; v < 2; v++) {
            d.a.src[v] = e.a.dst[v];
            d.a.dst[v] = pr[k].a.arms[v];
            d.a.rec[v] = pr[k].a.rec[v];
        }
        di.push_back(d);
    }
    if ((st = launch_items(h, s, "k_smooth", k_smooth<1, false>, k_smooth<kBatchMax, false>, er, 256, 0)) != DCO_OK)
        return st;
    return launch_items(h, s, "k_smooth", k_smooth<1, true>, k_smooth<kBatchMax, true>, di, 256, 0);
}

// pass `pass` (disparities [pass*dc, pass*dc + dc)) of every job that has it.
// Pairs are bucketed by block size (warps per block) so no block carries
// idle warps for a larger pair; one launch per bucket and stage.
// The slice of one view (dstride words per pixel, pixel index y * W + x) for
// the tile copies of k_vagg: a box of 36 words (the group's 32 disparities
// and 4 words of padding) by 32 consecutive rows (row_scan: columns).  Rank
// 4: dims (disparity within the group, group, x, y), the padding beyond the
// 32-long dimension 0 is zero-filled without a read.  Rank 3 (used if the
// encoder refuses a box wider than dimension 0): dims (disparity, x, y), the
// padding reads the next group's first words (zeros past the last group).
dco_status slice_map(dco_stereo *h, VArgs &a, int v, const uint32_t *slice, int W, int H, int dstride, bool row_scan)
{
    // the encoder's answer for rank 4, kept for the process (serving lanes
    // encode maps from several threads)
    static std::atomic<int> rank_seen{4};
    int rank = rank_seen.load(std::memory_order_relaxed);
    TmapEncode enc = tmap_encoder();
    if (!enc) {
        h->last_error = "cuTensorMapEncodeTiled is not available";
        return DCO_ECUDA;
    }
    const cuuint32_t rows = row_scan ? 1u : (cuuint32_t)kVSeg, cols = row_scan ? (cuuint32_t)kVSeg : 1u;
    const cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = CUDA_ERROR_INVALID_VALUE;
    if (rank == 4) {
        const cuuint64_t dims[4] = {32, (cuuint64_t)(dstride / 32), (cuuint64_t)W, (cuuint64_t)H};
        const cuuint64_t strides[3] = {128, (cuuint64_t)dstride * 4, (cuuint64_t)W * dstride * 4};
        const cuuint32_t box[4] = {(cuuint32_t)kQS, 1, cols, rows};
        r = enc(&a.tm[v], CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, const_cast<uint32_t *>(slice), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            rank = 3;
            rank_seen.store(3, std::memory_order_relaxed);
        }
    }
    if (rank == 3) {
        const cuuint64_t dims[3] = {(cuuint64_t)dstride, (cuuint64_t)W, (cuuint64_t)H};
        const cuuint64_t strides[2] = {(cuuint64_t)dstride * 4, (cuuint64_t)W * dstride * 4};
        const cuuint32_t box[3] = {(cuuint32_t)kQS, cols, rows};
        r = enc(&a.tm[v], CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, const_cast<uint32_t *>(slice), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS) {
        h->last_error = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
        return DCO_ECUDA;
    }
    a.tm_rank = rank;
    return DCO_OK;
}

// bounded tile waits of the V pass; the lost-copy failure test arms the
// barriers without copies and gives up after a few polls
void set_wait(const dco_stereo *h, VArgs &a)
{
    const bool lose = (h->test_flags & DCO_TEST_LOSE_TILE_COPIES) != 0;
    a.wait_limit = lose ? kTestWaitLimit : kWaitLimit;
    a.skip_copy = lose ? 1 : 0;
}

dco_status launch_pass(dco_stereo *h, const Derived &dv, const std::vector<Job> &jobs, int pass, cudaStream_t s)
{
    std::map<int, std::vector<Item<HArgs>>> hb;
    std::map<int, std::vector<Item<VArgs>>> vb;
    std::map<int, size_t> hsm, vsm;
    const bool vh = dv.order == 1;   // vertical segment sums first (k_vcost), then rows (k_vagg<.., kRow>)
    for (const Job &j : jobs) {
        if (pass >= j.L.npass) continue;
        const int d0 = dv.dmin + pass * j.L.dc, dc = std::min(j.L.dc, dv.dmin + j.D - d0);
        const int hw = j.hchunk > 0 ? j.hchunk : dv.hchunk, vw = j.vchunk > 0 ? j.vchunk : dv.vchunk;
        const HGeom hg = vh ? vcost_geom(j.W, j.H, dc, dv.L1, hw) : hagg_geom(j.W, j.H, dc, dv.L1, hw);
        const VGeom vg = vh ? vagg_geom(j.H, j.W, dv.L1, vw) : vagg_geom(j.W, j.H, dv.L1, vw);
        hsm[hg.nw] = std::max(hsm[hg.nw], hg.smem);
        vsm[vg.nw] = std::max(vsm[vg.nw], vg.smem);
        Item<HArgs> a{};
        for (int v = 0; v < 2; v++) {
            a.a.rec[v] = jptr<uint4>(h, j, j.L.rec[v]) + kRPad;
            a.a.cen[v] = jptr<uint2>(h, j, j.L.cen[v]);
            a.a.col[v] = jptr<uint32_t>(h, j, j.L.col[v]);
            a.a.arms[v] = jptr<uchar4>(h, j, j.L.arms[v]);
            a.a.sh[v] = jptr<uint32_t>(h, j, j.L.sh[v]);
        }
        a.a.phw = j.L.phw;
        a.a.status = h->d_status;
        {   // bounded staging waits; the lost-copy failure test arms the barrier without copies
            const bool lose = (h->test_flags & DCO_TEST_LOSE_TILE_COPIES) != 0;
            a.a.wait_limit = lose ? kTestWaitLimit : kWaitLimit;
            a.a.skip_copy = lose ? 1 : 0;
        }
        a.a.tables = h->d_tables;
        a.a.W = j.W; a.a.H = j.H; a.a.D = dv.dmin + j.D; a.a.rpitch = j.L.rpitch;
        a.a.d0 = d0; a.a.dc = dc; a.a.dstride = j.L.dstride;
        a.a.ngroups = (dc + 31) / 32;
        a.a.L1 = dv.L1; a.a.chunk = hg.chunk; a.a.S = dv.S; a.a.Sint = dv.Sint;
        a.gx = hg.grid.x; a.gy = hg.grid.y; a.gz = hg.grid.z;
        hb[hg.nw].push_back(a);
        Item<VArgs> b{};
        for (int v = 0; v < 2; v++) {
            b.a.sh[v] = a.a.sh[v];
            b.a.arms[v] = a.a.arms[v];
            b.a.best[v] = jptr<unsigned long long>(h, j, j.L.best[v]);
        }
        b.a.disp[0] = j.disp_l; b.a.disp[1] = j.disp_r;
        b.a.cost[0] = j.cost_l; b.a.cost[1] = j.cost_r;
        b.a.vol = j.vol; b.a.vol_view = j.vol_view;
        b.a.W = j.W; b.a.H = j.H; b.a.D = dv.dmin + j.D; b.a.dmin = dv.dmin;
        b.a.d0 = d0; b.a.dc = dc; b.a.dstride = j.L.dstride;
        b.a.first = pass == 0; b.a.last = pass == j.L.npass - 1;
        b.a.status = h->d_status; b.a.L1 = dv.L1; b.a.chunk = vg.chunk; b.a.seglog = vg.seglog; b.a.S = dv.S;
        set_wait(h, b.a);
        for (int v = 0; v < 2; v++) {
            dco_status st = slice_map(h, b.a, v, b.a.sh[v], j.W, j.H, j.L.dstride, vh);
            if (st != DCO_OK) return st;
        }
        b.gx = vg.grid.x; b.gy = vg.grid.y; b.gz = vg.grid.z;
        vb[vg.nw].push_back(b);
    }
    for (auto &kv : hb) {
        if (vh) {
            dco_status st = launch_items(h, s, "k_vcost", k_vcost<1>, k_vcost<kBatchMax>, kv.second, kv.first * 32,
                                         hsm[kv.first]);
            if (st != DCO_OK) return st;
            continue;
        }
        dco_status st = kv.first <= kHNarrow
                            ? launch_items(h, s, "k_hagg", k_hagg<1, false>, k_hagg<kBatchMax, false>, kv.second,
                                           kv.first * 32, hsm[kv.first])
                            : launch_items(h, s, "k_hagg", k_hagg<1, true>, k_hagg<kBatchMax, true>, kv.second,
                                           kv.first * 32, hsm[kv.first]);
        if (st != DCO_OK) return st;
    }
    for (auto &kv : vb) {
        dco_status st = vh ? launch_items(h, s, "k_hwta", k_vagg<1, false, true>, k_vagg<kVBatch, false, true>,
                                          kv.second, kv.first * 32, vsm[kv.first])
                           : launch_items(h, s, "k_vagg", k_vagg<1, false>, k_vagg<kVBatch, false>, kv.second,
                                          kv.first * 32, vsm[kv.first]);
        if (st != DCO_OK) return st;
    }
    return DCO_OK;
}

dco_status launch_lr(dco_stereo *h, const std::vector<Item<LrArgs>> &items, cudaStream_t s)
{
    return launch_items(h, s, "k_lr", k_lr<1>, k_lr<kBatchMax>, items, 256, 0);
}

// disparities [d0, d0 + dc) of pass `pass` of one Eq. 4 round, every job
// with a map to vote on: vote counts per horizontal segment (k_hvote), then
// vertical sums and the count maximum (k_vagg in vote mode, "k_vvote")
dco_status launch_vote_pass(dco_stereo *h, const Derived &dv, const std::vector<Job> &jobs, int pass,
                            cudaStream_t s)
{
    std::map<int, std::vector<Item<HVArgs>>> hb;
    std::map<int, std::vector<Item<VArgs>>> vb;
    std::map<int, size_t> hsm, vsm;
    for (const Job &j : jobs) {
        if (!j.vsrc || pass >= j.L.npass) continue;
        const int d0 = dv.dmin + pass * j.L.dc, dc = std::min(j.L.dc, dv.dmin + j.D - d0);
        const int hw = j.hchunk > 0 ? j.hchunk : dv.hchunk, vw = j.vchunk > 0 ? j.vchunk : dv.vchunk;
        const HGeom hg = hagg_geom(j.W, j.H, dc, dv.L1, hw);
        const VGeom vg = vagg_geom(j.W, j.H, dv.L1, vw);
        const int hlen = std::min(j.W, hg.chunk + 2 * dv.L1), vlen = std::min(j.H, vg.chunk + 2 * dv.L1);
        const int hnw = (hlen + kHSeg - 1) / kHSeg;   // the vote pass walks 64-column segments
        hsm[hnw] = std::max(hsm[hnw], (size_t)HVSmem(hlen, hg.chunk, hnw).total);
        vsm[vg.nw] = std::max(vsm[vg.nw], vagg_smem_words(vlen, vg.nw) * 4);
        Item<HVArgs> a{};
        a.a.disp = j.vsrc;
        a.a.arms = jptr<uchar4>(h, j, j.L.arms[0]);
        a.a.sh = jptr<uint32_t>(h, j, j.L.sh[0]);
        a.a.W = j.W; a.a.H = j.H; a.a.d0 = d0; a.a.dstride = j.L.dstride;
        a.a.L1 = dv.L1; a.a.chunk = hg.chunk;
        a.gx = hg.grid.x; a.gy = hg.grid.y; a.gz = (dc + 31) / 32;
        hb[hnw].push_back(a);
        Item<VArgs> b{};
        for (int v = 0; v < 2; v++) {
            b.a.sh[v] = a.a.sh;
            b.a.arms[v] = a.a.arms;
            b.a.best[v] = jptr<unsigned long long>(h, j, j.L.best[0]);
            b.a.disp[v] = j.vdst;
        }
        b.a.mask = j.vsrc;
        b.a.W = j.W; b.a.H = j.H; b.a.D = dv.dmin + j.D; b.a.dmin = dv.dmin;
        b.a.d0 = d0; b.a.dc = dc; b.a.dstride = j.L.dstride;
        b.a.first = pass == 0; b.a.last = pass == j.L.npass - 1;
        b.a.status = h->d_status; b.a.L1 = dv.L1; b.a.chunk = vg.chunk; b.a.seglog = vg.seglog; b.a.S = dv.S;
        set_wait(h, b.a);
        if (dco_status st = slice_map(h, b.a, 0, b.a.sh[0], j.W, j.H, j.L.dstride, false); st != DCO_OK) return st;
        b.a.tm[1] = b.a.tm[0];
        b.gx = vg.grid.x; b.gy = 1; b.gz = vg.grid.z;   // the left view only
        vb[vg.nw].push_back(b);
    }
    for (auto &kv : hb) {
        dco_status st = launch_items(h, s, "k_hvote", k_hvote<1>, k_hvote<kBatchMax>, kv.second, kv.first * 32,
                                     hsm[kv.first]);
        if (st != DCO_OK) return st;
    }
    for (auto &kv : vb) {
        dco_status st = launch_items(h, s, "k_vvote", k_vagg<1, true>, k_vagg<kVBatch, true>, kv.second,
                                     kv.first * 32, vsm[kv.first]);
        if (st != DCO_OK) return st;
    }
    return DCO_OK;
}

// p.vote_iters rounds of Eq. 4 on every job's final map (j.out, in place),
// alternating with the job's second map; arms of the left view in the
// workspace
dco_status run_vote(dco_stereo *h, const dco_params &p, const Derived &dv, std::vector<Job> &jobs, cudaStream_t s)
{
    int maxpass = 0;
    for (const Job &j : jobs) maxpass = std::max(maxpass, j.L.npass);
    for (int it = 0; it < p.vote_iters; it++) {
        for (Job &j : jobs) {
            int16_t *tmp = jptr<int16_t>(h, j, j.L.vtmp);
            j.vsrc = !j.out ? nullptr : (it & 1) ? tmp : j.out;
            j.vdst = (it & 1) ? j.out : tmp;
        }
        for (int pass = 0; pass < maxpass; pass++) {
            dco_status st = launch_vote_pass(h, dv, jobs, pass, s);
            if (st != DCO_OK) return st;
        }
    }
    if (p.vote_iters & 1)
        for (const Job &j : jobs)
            if (j.out)
                DCO_CUDA(h, cudaMemcpyAsync(j.out, jptr<int16_t>(h, j, j.L.vtmp), sizeof(int16_t) * j.W * j.H,
                                            cudaMemcpyDeviceToDevice, s));
    return DCO_OK;
}

// every stage of the path for planned jobs (workspace and tables ready)
dco_status launch_jobs(dco_stereo *h, const dco_params &p, const Derived &dv, std::vector<Job> &jobs,
                       cudaStream_t s)
{
    int maxpass = 0;
    for (Job &j : jobs) {
        if (!j.disp_l) j.disp_l = jptr<int16_t>(h, j, j.L.disp[0]);
        if (!j.disp_r) j.disp_r = jptr<int16_t>(h, j, j.L.disp[1]);
        maxpass = std::max(maxpass, j.L.npass);
    }
    dco_status st;
    if ((st = launch_prep(h, p, dv, jobs, 2, s)) != DCO_OK) return st;
    for (int pass = 0; pass < maxpass; pass++)
        if ((st = launch_pass(h, dv, jobs, pass, s)) != DCO_OK) return st;
    std::vector<Item<LrArgs>> lr;
    for (const Job &j : jobs) {
        if (!j.out) continue;
        Item<LrArgs> it{};
        it.a.dl = j.disp_l; it.a.dr = j.disp_r; it.a.out = j.out;
        it.a.W = j.W; it.a.H = j.H; it.a.tol = p.lr_tol;
        it.gx = (j.W * j.H + 255) / 256; it.gy = 1; it.gz = 1;
        lr.push_back(it);
    }
    if ((st = launch_lr(h, lr, s)) != DCO_OK) return st;
    return p.vote_iters > 0 ? run_vote(h, p, dv, jobs, s) : DCO_OK;
}

// the whole path for a set of independent pairs: one launch per stage.  On a
// handle with a budget, pairs whose workspaces do not fit it together (even
// at the narrowest pass width) are admitted in consecutive groups that do;
// the groups run one after the other on the stream, each reusing the same
// workspace.  Every group is planned before anything is enqueued.
dco_status run_jobs(dco_stereo *h, const dco_params &p, std::vector<Job> &jobs, cudaStream_t s)
{
    Derived dv;
    derive(p, dv);
    size_t total = 0;
    dco_status st = plan_jobs(h, p, jobs, total);
    if (st != DCO_OK) return st;
    if (!h->budget || total <= h->budget || jobs.size() == 1) {
        if ((st = ensure_ws(h, total)) != DCO_OK) return st;
        if ((st = ensure_tables(h, p, dv, s)) != DCO_OK) return st;
        return launch_jobs(h, p, dv, jobs, s);
    }
    std::vector<std::vector<Job>> groups;
    size_t need = 0;
    for (size_t i = 0; i < jobs.size();) {
        std::vector<Job> g{jobs[i]};
        size_t t = 0;
        plan_jobs(h, p, g, t);
        if (t > h->budget) {
            h->last_error = "pair " + std::to_string(i) + " needs " + std::to_string(t) +
                            " bytes of workspace, more than the budget of " + std::to_string(h->budget);
            return DCO_EBUDGET;
        }
        size_t j = i + 1;
        for (; j < jobs.size(); j++) {
            std::vector<Job> g2 = g;
            g2.push_back(jobs[j]);
            size_t t2 = 0;
            plan_jobs(h, p, g2, t2);
            if (t2 > h->budget) break;
            g.swap(g2);
            t = t2;
        }
        need = std::max(need, t);
        groups.push_back(std::move(g));
        i = j;
    }
    if ((st = ensure_ws(h, need)) != DCO_OK) return st;
    if ((st = ensure_tables(h, p, dv, s)) != DCO_OK) return st;
    h->groups_last = (int)groups.size();
    for (auto &g : groups)
        if ((st = launch_jobs(h, p, dv, g, s)) != DCO_OK) return st;
    return DCO_OK;
}

dco_status check_common(dco_stereo *h, const dco_params *pin, dco_params &p)
{
    if (!h) return DCO_EINVAL;
    if (pin) p = *pin;
    else dco_params_default(&p);
    if (!params_valid(p)) {
        h->last_error = "invalid parameters";
        return DCO_EINVAL;
    }
    DCO_CUDA(h, enter_device(h));
    return DCO_OK;
}

dco_status run_match(dco_stereo *h, const uint8_t *left, const uint8_t *right, int W, int H, int D,
                     const dco_params &p, int16_t *disp_out, int16_t *disp_l, int16_t *disp_r,
                     float *cost_l, float *cost_r, float *vol, int vol_view, cudaStream_t s, int host_in = -1)
{
    std::vector<Job> jobs(1);
    Job &j = jobs[0];
    j.left = left; j.right = right; j.W = W; j.H = H; j.D = D;
    j.host_in = host_in;
    j.out = disp_out; j.disp_l = disp_l; j.disp_r = disp_r;
    j.cost_l = cost_l; j.cost_r = cost_r; j.vol = vol; j.vol_view = vol_view;
    return run_jobs(h, p, jobs, s);
}

} // namespace

// ===================================================================== C ABI
#include "densify.cuh"

extern "C" {

dco_status dco_params_default(dco_params *p)
{
    if (!p) return DCO_EINVAL;
    p->lambda_ad = 10.0f;
    p->lambda_census = 40.0f;
    p->gamma_l = 1.0f;
    p->eps = 0.8f;
    p->census_w = 9;
    p->census_h = 7;
    p->arm_l1 = 34;
    p->arm_l2 = 17;
    p->tau1 = 20;
    p->tau2 = 6;
    p->lr_tol = 1;
    p->d_chunk = 0;
    p->vote_iters = 0;
    p->smooth_arms = 0;
    p->agg_order = 0;
    p->d_min = 0;
    p->h_chunk = 0;
    p->v_chunk = 0;
    return DCO_OK;
}

const char *dco_status_string(dco_status s)
{
    switch (s) {
    case DCO_OK: return "ok";
    case DCO_EINVAL: return "invalid argument";
    case DCO_ENOMEM: return "device allocation failed";
    case DCO_EBUDGET: return "workspace budget exceeded";
    case DCO_ECUDA: return "CUDA runtime error";
    case DCO_ETIMEOUT: return "device-side wait timed out";
    case DCO_EDEVICE: return "kernel reported a failed internal check";
    }
    return "unknown status";
}

dco_status dco_stereo_create(dco_stereo **out, int device, size_t workspace_budget_bytes)
{
    if (!out) return DCO_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return DCO_EINVAL;
    dco_stereo *h = new (std::nothrow) dco_stereo();
    if (!h) return DCO_ENOMEM;
    h->device = device;
    h->budget = workspace_budget_bytes;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_tables, sizeof(float) * kTabFloats);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->h_tables, sizeof(float) * kTabFloats);
    if (e != cudaSuccess) {
        dco_stereo_destroy(h);
        return e == cudaErrorMemoryAllocation ? DCO_ENOMEM : DCO_ECUDA;
    }
    *out = h;
    return DCO_OK;
}

void dco_stereo_destroy(dco_stereo *h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    for (auto &pe : h->pending) { cudaEventDestroy(pe.a); cudaEventDestroy(pe.b); }
    for (auto e : h->pool) cudaEventDestroy(e);
    cudaFree(h->ws);
    cudaFree(h->d_status);
    cudaFree(h->d_tables);
    cudaFree(h->stage);
    if (h->h_tables) cudaFreeHost(h->h_tables);
    if (h->dn_pin) cudaFreeHost(h->dn_pin);
    if (h->dn_exec) cudaGraphExecDestroy(h->dn_exec);
    if (h->dn_stream) cudaStreamDestroy(h->dn_stream);
    for (auto e : h->dn_ev)
        if (e) cudaEventDestroy(e);
    delete h;
}

size_t dco_stereo_workspace_bytes(int W, int H, int D, const dco_params *pin)
{
    dco_params p;
    if (pin) p = *pin;
    else dco_params_default(&p);
    if (!params_valid(p) || !dims_valid(W, H, D, p.d_min)) return 0;
    return make_layout(W, H, D, p).total;
}

dco_status dco_stereo_reserve(dco_stereo *h, int W, int H, int D, const dco_params *pin)
{
    dco_params p;
    dco_status st = check_common(h, pin, p);
    if (st != DCO_OK) return st;
    if (!dims_valid(W, H, D, p.d_min)) return DCO_EINVAL;
    return ensure_ws(h, make_layout(W, H, D, p).total);
}

dco_status dco_stereo_match_views(dco_stereo *h, const uint8_t *left, const uint8_t *right, int W, int H,
                                  int D, const dco_params *pin, int16_t *disp_out, int16_t *disp_left,
                                  int16_t *disp_right, float *cost_left, float *cost_right,
                                  dco_stream stream)
{
    dco_params p;
    dco_status st = check_common(h, pin, p);
    if (st != DCO_OK) return st;
    if (!left || !right || !dims_valid(W, H, D, p.d_min)) return DCO_EINVAL;
    return run_match(h, left, right, W, H, D, p, disp_out, disp_left, disp_right, cost_left, cost_right,
                     nullptr, 0, (cudaStream_t)stream);
}

dco_status dco_stereo_match(dco_stereo *h, const uint8_t *left, const uint8_t *right, int W, int H, int D,
                            const dco_params *p, int16_t *disp_out, dco_stream stream)
{
    if (!disp_out) return DCO_EINVAL;
    return dco_stereo_match_views(h, left, right, W, H, D, p, disp_out, nullptr, nullptr, nullptr, nullptr,
                                  stream);
}

// the device can dereference p at the same address (pinned, registered or
// managed host memory)
static bool device_accessible(const void *p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();   // plain pageable memory: not an error for the caller
        return false;
    }
    return (at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeManaged) && at.devicePointer == p;
}

dco_status dco_stereo_match_host(dco_stereo *h, const uint8_t *left_host, const uint8_t *right_host, int W,
                                 int H, int D, const dco_params *pin, int16_t *disp_host, dco_stream stream)
{
    dco_params p;
    dco_status st = check_common(h, pin, p);
    if (st != DCO_OK) return st;
    if (!left_host || !right_host || !disp_host || !dims_valid(W, H, D, p.d_min)) return DCO_EINVAL;
    const size_t img = (size_t)W * H * 3, out = (size_t)W * H * 2;
    const size_t need = align_up(img) * 2 + align_up(out);
    cudaStream_t s = (cudaStream_t)stream;
    // Buffers the device can dereference (pinned, registered or managed host
    // memory; over NVLink-C2C on Grace systems) are read by k_pack and
    // written by the consistency check in place, without staging copies.
    // With Eq. 4 rounds the map is rewritten several times: it stays on the
    // device and is copied once.
    if (device_accessible(left_host) && device_accessible(right_host) && device_accessible(disp_host) &&
        p.vote_iters == 0) {
        st = run_match(h, left_host, right_host, W, H, D, p, disp_host, nullptr, nullptr, nullptr, nullptr, nullptr,
                       0, s, 1);
        if (st != DCO_OK) return st;
        DCO_CUDA(h, cudaStreamSynchronize(s));
        return DCO_OK;
    }
    if (h->stage_cap < need) {
        if (h->stage) {
            DCO_CUDA(h, cudaDeviceSynchronize());
            cudaFree(h->stage);
            h->stage = nullptr;
            h->stage_cap = 0;
        }
        DCO_CUDA(h, cudaMalloc((void **)&h->stage, need));
        h->stage_cap = need;
    }
    uint8_t *dl = h->stage, *dr = h->stage + align_up(img);
    int16_t *dd = reinterpret_cast<int16_t *>(h->stage + 2 * align_up(img));
    DCO_CUDA(h, cudaMemcpyAsync(dl, left_host, img, cudaMemcpyHostToDevice, s));
    DCO_CUDA(h, cudaMemcpyAsync(dr, right_host, img, cudaMemcpyHostToDevice, s));
    st = run_match(h, dl, dr, W, H, D, p, dd, nullptr, nullptr, nullptr, nullptr, nullptr, 0, s);
    if (st != DCO_OK) return st;
    DCO_CUDA(h, cudaMemcpyAsync(disp_host, dd, out, cudaMemcpyDeviceToHost, s));
    DCO_CUDA(h, cudaStreamSynchronize(s));
    return DCO_OK;
}

// census + arms of one image (stage entry points): the pack/prep launches
// of a one-job run with a single image
static dco_status prep_one(dco_stereo *h, const dco_params &p, const uint8_t *rgb, int W, int H,
                           uchar4 *arms_out, std::vector<Job> &jobs, cudaStream_t s)
{
    Derived dv;
    derive(p, dv);
    jobs.assign(1, Job{});
    Job &j = jobs[0];
    j.left = rgb; j.right = rgb; j.W = W; j.H = H; j.D = 1; j.arms0 = arms_out;
    size_t total = 0;
    dco_status st = plan_jobs(h, p, jobs, total);
    if (st != DCO_OK) return st;
    if ((st = ensure_ws(h, total)) != DCO_OK) return st;
    if ((st = ensure_tables(h, p, dv, s)) != DCO_OK) return st;
    return launch_prep(h, p, dv, jobs, 1, s);
}

dco_status dco_stereo_census(dco_stereo *h, const uint8_t *rgb, int W, int H, const dco_params *pin,
                             uint64_t *census_out, dco_stream stream)
{
    dco_params p;
    dco_status st = check_common(h, pin, p);
    if (st != DCO_OK) return st;
    if (!rgb || !census_out || !dims_valid(W, H, 1)) return DCO_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<Job> jobs;
    if ((st = prep_one(h, p, rgb, W, H, nullptr, jobs, s)) != DCO_OK) return st;
    const Job &j = jobs[0];
    const size_t n = (size_t)W * H;
    ProfScope ps(h, s, "k_extract_census");
    k_extract_census<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(jptr<uint4>(h, j, j.L.rec[0]) + kRPad, W, H,
                                                                  j.L.rpitch,
                                                                  reinterpret_cast<unsigned long long *>(census_out));
    DCO_CUDA(h, cudaGetLastError());
    return DCO_OK;
}

dco_status dco_stereo_arms(dco_stereo *h, const uint8_t *rgb, int W, int H, const dco_params *pin,
                           uint8_t *arms_out, dco_stream stream)
{
    dco_params p;
    dco_status st = check_common(h, pin, p);
    if (st != DCO_OK) return st;
    if (!rgb || !arms_out || !dims_valid(W, H, 1)) return DCO_EINVAL;
    std::vector<Job> jobs;
    return prep_one(h, p, rgb, W, H, reinterpret_cast<uchar4 *>(arms_out), jobs, (cudaStream_t)stream);
}

dco_status dco_stereo_vote(dco_stereo *h, const uint8_t *rgb, const int16_t *disp_in, int W, int H, int D,
                           const dco_params *pin, int16_t *disp_out, dco_stream stream)
{
    dco_params p;
    dco_status st = check_common(h, pin, p);
    if (st != DCO_OK) return st;
    if (!rgb || !disp_in || !disp_out || !dims_valid(W, H, D, p.d_min)) return DCO_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Derived dv;
    derive(p, dv);
    std::vector<Job> jobs(1);
    Job &j = jobs[0];
    j.left = rgb; j.right = rgb; j.W = W; j.H = H; j.D = D; j.out = disp_out;
    size_t total = 0;
    if ((st = plan_jobs(h, p, jobs, total)) != DCO_OK) return st;
    if ((st = ensure_ws(h, total)) != DCO_OK) return st;
    if ((st = ensure_tables(h, p, dv, s)) != DCO_OK) return st;
    if ((st = launch_prep(h, p, dv, jobs, 1, s)) != DCO_OK) return st;   // arms of rgb
    if (disp_in != disp_out)
        DCO_CUDA(h, cudaMemcpyAsync(disp_out, disp_in, sizeof(int16_t) * W * H, cudaMemcpyDeviceToDevice, s));
    return run_vote(h, p, dv, jobs, s);
}

dco_status dco_stereo_downscale(dco_stereo *h, const uint8_t *rgb, int W, int H, uint8_t *out, dco_stream stream)
{
    if (!h || !rgb || !out || W < 2 || H < 2 || W > 2 * 16384 || H > 2 * 16384) return DCO_EINVAL;
    DCO_CUDA(h, enter_device(h));
    cudaStream_t s = (cudaStream_t)stream;
    DownArgs da{};
    da.src[0] = rgb; da.dst[0] = out; da.W = W; da.H = H;
    ProfScope ps(h, s, "k_down");
    launch_pdl(k_down, dim3((unsigned)((W / 2 + 255) / 256), (unsigned)(H / 2), 1), dim3(256), 0, s, da);
    DCO_CUDA(h, cudaGetLastError());
    return DCO_OK;
}

dco_status dco_stereo_depth(dco_stereo *h, const uint8_t *left, const uint8_t *right, int W, int H, int D,
                            const dco_params *pin, double f_px, double baseline, float *depth_out,
                            int16_t *disp_half_out, dco_stream stream)
{
    dco_params p;
    dco_status st = check_common(h, pin, p);
    if (st != DCO_OK) return st;
    if (!left || !right || !depth_out || W < 2 || H < 2 || !dims_valid(W / 2, H / 2, D, p.d_min)) return DCO_EINVAL;
    if (!(f_px > 0.0) || !(baseline > 0.0) || !std::isfinite(f_px * baseline)) return DCO_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int Wh = W / 2, Hh = H / 2;
    Derived dv;
    derive(p, dv);
    std::vector<Job> jobs(1);
    Job &j = jobs[0];
    j.W = Wh; j.H = Hh; j.D = D;
    size_t total = 0;
    if ((st = plan_jobs(h, p, jobs, total)) != DCO_OK) return st;
    // in front of the pair's workspace: the two half-size images and the map
    const size_t img = align_up(3 * (size_t)Wh * Hh), front = 2 * img + align_up(2 * (size_t)Wh * Hh);
    j.base = front;
    if ((st = ensure_ws(h, total + front)) != DCO_OK) return st;
    if ((st = ensure_tables(h, p, dv, s)) != DCO_OK) return st;
    DownArgs da{};
    da.src[0] = left; da.src[1] = right;
    da.dst[0] = ws_ptr<uint8_t>(h, 0); da.dst[1] = ws_ptr<uint8_t>(h, img);
    da.W = W; da.H = H;
    j.left = da.dst[0]; j.right = da.dst[1];
    j.out = disp_half_out ? disp_half_out : ws_ptr<int16_t>(h, 2 * img);
    {
        ProfScope ps(h, s, "k_down");
        launch_pdl(k_down, dim3((unsigned)((Wh + 255) / 256), (unsigned)Hh, 2), dim3(256), 0, s, da);
        DCO_CUDA(h, cudaGetLastError());
    }
    if ((st = launch_jobs(h, p, dv, jobs, s)) != DCO_OK) return st;
    DepthArgs za{};
    za.disp = j.out; za.out = depth_out; za.W = W; za.H = H; za.fb = (float)(f_px * baseline);
    ProfScope ps(h, s, "k_depth");
    launch_pdl(k_depth, dim3((unsigned)(((W + 1) / 2 + 255) / 256), (unsigned)((H + 1) / 2)), dim3(256), 0, s, za);
    DCO_CUDA(h, cudaGetLastError());
    return DCO_OK;
}

dco_status dco_stereo_cost_volume(dco_stereo *h, const uint8_t *left, const uint8_t *right, int W, int H,
                                  int D, const dco_params *pin, int view, float *vol_out, dco_stream stream)
{
    dco_params p;
    dco_status st = check_common(h, pin, p);
    if (st != DCO_OK) return st;
    if (!left || !right || !vol_out || (view != 0 && view != 1) || !dims_valid(W, H, D, p.d_min)) return DCO_EINVAL;
    return run_match(h, left, right, W, H, D, p, nullptr, nullptr, nullptr, nullptr, nullptr, vol_out, view,
                     (cudaStream_t)stream);
}

dco_status dco_stereo_lr_check(dco_stereo *h, const int16_t *dl, const int16_t *dr, int W, int H, int tol,
                               int16_t *out, dco_stream stream)
{
    if (!h || !dl || !dr || !out || W < 1 || H < 1) return DCO_EINVAL;
    DCO_CUDA(h, enter_device(h));
    std::vector<Item<LrArgs>> it(1);
    it[0].a.dl = dl; it[0].a.dr = dr; it[0].a.out = out;
    it[0].a.W = W; it[0].a.H = H; it[0].a.tol = tol;
    it[0].gx = (int)(((size_t)W * H + 255) / 256); it[0].gy = 1; it[0].gz = 1;
    return launch_lr(h, it, (cudaStream_t)stream);
}

dco_status dco_stereo_match_batch(dco_stereo *h, const dco_pair_desc *descs, int n, const dco_params *pin,
                                  dco_stream stream)
{
    dco_params p;
    dco_status st = check_common(h, pin, p);
    if (st != DCO_OK) return st;
    h->groups_last = 1;
    if (n < 0 || (n > 0 && !descs)) return DCO_EINVAL;
    for (int i = 0; i < n; i++)
        if (!descs[i].left || !descs[i].right || !descs[i].disp_out ||
            !dims_valid(descs[i].W, descs[i].H, descs[i].D, p.d_min) || descs[i].d_chunk < 0 ||
            !tile_valid(descs[i].h_chunk) || !tile_valid(descs[i].v_chunk))
            return DCO_EINVAL;
    if (n == 0) return DCO_OK;
    std::vector<Job> jobs(n);
    for (int i = 0; i < n; i++) {
        jobs[i].left = descs[i].left; jobs[i].right = descs[i].right;
        jobs[i].W = descs[i].W; jobs[i].H = descs[i].H; jobs[i].D = descs[i].D;
        jobs[i].out = descs[i].disp_out;
        jobs[i].dchunk = descs[i].d_chunk;
        jobs[i].hchunk = descs[i].h_chunk;
        jobs[i].vchunk = descs[i].v_chunk;
    }
    return run_jobs(h, p, jobs, (cudaStream_t)stream);
}

dco_status dco_stereo_sync_status(dco_stereo *h)
{
    if (!h) return DCO_EINVAL;
    DCO_CUDA(h, enter_device(h));
    DCO_CUDA(h, cudaDeviceSynchronize());
    int v = 0;
    DCO_CUDA(h, cudaMemcpy(&v, h->d_status, sizeof v, cudaMemcpyDeviceToHost));
    DCO_CUDA(h, cudaMemset(h->d_status, 0, sizeof v));
    return status_of_word(v);
}

dco_status dco_stereo_stream_status(dco_stereo *h, dco_stream stream)
{
    if (!h) return DCO_EINVAL;
    DCO_CUDA(h, enter_device(h));
    const cudaStream_t s = (cudaStream_t)stream;
    // a device-to-pageable copy returns once it has completed: the word is
    // read after everything enqueued on `stream` before this call
    int v = 0;
    DCO_CUDA(h, cudaMemcpyAsync(&v, h->d_status, sizeof v, cudaMemcpyDeviceToHost, s));
    DCO_CUDA(h, cudaStreamSynchronize(s));
    DCO_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof v, s));
    return status_of_word(v);
}

dco_status dco_stereo_set_test_flags(dco_stereo *h, int flags)
{
    if (!h || (flags & ~(DCO_TEST_LOSE_TILE_COPIES | DCO_TEST_LOSE_GRID_ARRIVAL))) return DCO_EINVAL;
    h->test_flags = flags;
    return DCO_OK;
}

size_t dco_stereo_workspace_allocated(dco_stereo *h)
{
    return h ? h->ws_cap : 0;
}

int dco_stereo_batch_groups(dco_stereo *h)
{
    return h ? h->groups_last : 0;
}

dco_status dco_stereo_set_profiling(dco_stereo *h, int enable)
{
    if (!h) return DCO_EINVAL;
    h->profiling = enable != 0;
    return DCO_OK;
}

dco_status dco_stereo_profile_reset(dco_stereo *h)
{
    if (!h) return DCO_EINVAL;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    collect_profile(h);
    h->agg.clear();
    return DCO_OK;
}

int dco_stereo_profile_count(dco_stereo *h)
{
    if (!h) return 0;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    collect_profile(h);
    return (int)h->agg.size();
}

dco_status dco_stereo_profile_get(dco_stereo *h, int i, const char **name, int *launches, double *total_ms)
{
    if (!h || i < 0 || i >= (int)h->agg.size()) return DCO_EINVAL;
    if (name) *name = h->agg[i].name.c_str();
    if (launches) *launches = h->agg[i].launches;
    if (total_ms) *total_ms = h->agg[i].ms;
    return DCO_OK;
}

unsigned long long dco_stereo_launch_count(dco_stereo *h)
{
    return h ? h->launches : 0ull;
}

const char *dco_stereo_last_error(dco_stereo *h)
{
    return h ? h->last_error.c_str() : "null handle";
}

} // extern "C"

// ======================================================= no-allocation entry
// For callers that may not allocate device memory: the scratch lives in one
// file-scope device array that every GPU loading this library holds until
// exit.  Host code never uses the array's name as a device address: each
// device's address comes from cudaGetSymbolAddress, taken once per device
// on the first call with that device current.
namespace {
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
constexpr int kNoAllocMaxDevices = 64;
// scratch layout: the Eq. 1 tables, the status word, the workspace
constexpr size_t kNoAllocTabBytes = (sizeof(float) * kTabFloats + kAlign - 1) / kAlign * kAlign;
constexpr size_t kNoAllocStatusBytes = kAlign;
std::mutex g_noalloc_mu;
void *g_noalloc_base[kNoAllocMaxDevices] = {};

// the tables travel by value in the kernel parameters, so no host buffer
// has to outlive the call
struct TabBlock {
    float t[kTabFloats];
};
__global__ void k_put_tables(const __grid_constant__ TabBlock b, float *dst)
{
    for (int i = threadIdx.x; i < kTabFloats; i += blockDim.x) dst[i] = b.t[i];
}
} // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
dco_status noalloc_base(int dev, void **out)
{
    if (dev < 0 || dev >= kNoAllocMaxDevices) return DCO_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DCO_ECUDA;
        g_noalloc_base[dev] = p;
    }
    *out = g_noalloc_base[dev];
    return DCO_OK;
}
} // namespace

extern "C" dco_status dco_stereo_match_noalloc(const uint8_t *left, const uint8_t *right, int W, int H, int D,
                                               const dco_params *pin, int16_t *disp_out, dco_stream stream)
{
    dco_params p;
    if (pin) p = *pin;
    else dco_params_default(&p);
    if (!params_valid(p) || !left || !right || !disp_out || !dims_valid(W, H, D, p.d_min)) return DCO_EINVAL;
    p.d_chunk = 32;   // passes of 32 disparities keep the slices small
    Derived dv;
    derive(p, dv);
    const Layout L = make_layout(W, H, D, p);
    if (kNoAllocTabBytes + kNoAllocStatusBytes + L.total > kNoAllocScratchBytes) return DCO_EBUDGET;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DCO_ECUDA;
    (void)cudaGetLastError();   // an earlier call's error is not this call's launch failure
    void *base = nullptr;
    dco_status st = noalloc_base(dev, &base);
    if (st != DCO_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;

    // Eq. 1 tables (host double, rounded once to float) into the scratch
    TabBlock tb;
    fill_tables(tb.t, p, dv);
    k_put_tables<<<1, 256, 0, s>>>(tb, static_cast<float *>(base));
    if (cudaGetLastError() != cudaSuccess) return DCO_ECUDA;

    // a handle that owns nothing: its workspace and tables are the scratch
    dco_stereo view;
    view.device = dev;
    view.d_status = reinterpret_cast<int *>(static_cast<char *>(base) + kNoAllocTabBytes);
    view.ws = static_cast<char *>(base) + kNoAllocTabBytes + kNoAllocStatusBytes;
    view.ws_cap = kNoAllocScratchBytes - kNoAllocTabBytes - kNoAllocStatusBytes;
    view.d_tables = static_cast<float *>(base);
    view.tab_valid = true;
    view.tab_key[0] = p.lambda_ad;
    view.tab_key[1] = p.lambda_census;
    view.tab_key[2] = p.gamma_l;
    view.tab_key[3] = p.eps;
    view.tab_l1 = p.arm_l1;
    st = run_match(&view, left, right, W, H, D, p, disp_out, nullptr, nullptr, nullptr, nullptr, nullptr, 0, s);
    view.ws = nullptr;
    view.d_tables = nullptr;
    view.d_status = nullptr;
    return st;
}

extern "C" dco_status dco_stereo_noalloc_status(dco_stream stream)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DCO_ECUDA;
    void *base = nullptr;
    dco_status st = noalloc_base(dev, &base);
    if (st != DCO_OK) return st;
    int *word = reinterpret_cast<int *>(static_cast<char *>(base) + kNoAllocTabBytes);
    const cudaStream_t s = (cudaStream_t)stream;
    // a device-to-pageable copy returns once it has completed, after the
    // work enqueued on `stream` before it
    int v = 0;
    if (cudaMemcpyAsync(&v, word, sizeof v, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess || cudaMemsetAsync(word, 0, sizeof v, s) != cudaSuccess) {
        (void)cudaGetLastError();
        return DCO_ECUDA;
    }
    return status_of_word(v);
}

// ====================================================== serving runtime
#include "serve.cuh"
