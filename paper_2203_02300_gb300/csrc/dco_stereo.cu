// GB300 (sm_103a) AD-census stereo matcher: kernels and C ABI.
//
// Method: arXiv 2203.02300, Sect. 4 (census + AD cost with adaptive weight,
// Eq. 1; cross-support region aggregation, Eq. 2; winner-take-all, Eq. 3;
// outlier removal by left-right consistency, Sect. 4.3).
//
// Pipeline per pair (one stream, no host round trip):
//   k_prep   grey + census (shared-memory window) + four arms (shared-memory
//            cross tile) for both images -> 16-byte records + arm words
//   per pass of dc disparities:
//     k_hagg  Eq. 1 cost in fixed point, running row prefix in registers,
//             a 2*L1+2 deep ring of prefixes per lane in shared memory, and
//             the horizontal segment sum of every pixel -> sh slice
//     k_vagg  running column prefix of sh, the same ring along y, the
//             vertical sum over the up/down arms (Eq. 2), WTA (Eq. 3) by a
//             warp min-reduction, merged with the previous passes
//   k_lr     left-right consistency -> disparity map
// Lanes of a warp always hold consecutive disparities of one pixel: the
// record of the reference pixel is a broadcast load, the 32 candidates are
// consecutive records, ring accesses hit 32 distinct banks, and the slices
// are written and read as 128-byte lines.
#include "kernels.cuh"
#include "dco_stereo.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

namespace dco {

// ------------------------------------------------------------------ k_pack
// RGB (3 bytes per pixel) -> packed 32-bit colour and the integer grey level
// of the census, for both images; four pixels (12 bytes) per thread.
__device__ __forceinline__ uint32_t grey_of(uint32_t c)
{
    return (77u * (c & 0xffu) + 150u * ((c >> 8) & 0xffu) + 29u * ((c >> 16) & 0xffu) + 128u) >> 8;
}

__global__ void k_pack(PackArgs a)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;   // pixels 4q .. 4q+3
    const int i0 = 4 * q;
    if (i0 >= a.npx) return;
    const uint8_t *rgb = blockIdx.y ? a.rgb[1] : a.rgb[0];
    uint32_t *rgbx = blockIdx.y ? a.rgbx[1] : a.rgbx[0];
    uint8_t *grey = blockIdx.y ? a.grey[1] : a.grey[0];
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
    if (i0 + 4 <= a.npx) {
        *reinterpret_cast<uint4 *>(rgbx + i0) = make_uint4(c[0], c[1], c[2], c[3]);
        *reinterpret_cast<uint32_t *>(grey + i0) =
            grey_of(c[0]) | (grey_of(c[1]) << 8) | (grey_of(c[2]) << 16) | (grey_of(c[3]) << 24);
    } else {
        for (int k = 0; i0 + k < a.npx; k++) {
            rgbx[i0 + k] = c[k];
            grey[i0 + k] = (uint8_t)grey_of(c[k]);
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

// any colour channel of |a - b| >= t, t4 = t replicated in four bytes (t <= 255)
__device__ __forceinline__ bool any_ge(uint32_t a, uint32_t b, uint32_t t4)
{
    return (__vcmpgeu4(__vabsdiffu4(a, b), t4) & 0x00ffffffu) != 0u;
}

// 4 flags f_i = [byte_i(w) < c] -> bits f0 | f1<<1 | f2<<2 | f3<<3
__device__ __forceinline__ uint32_t lt4(uint32_t w, uint32_t c4)
{
    return (__vsetltu4(w, c4) * 0x01020408u) >> 24;
}

template <int CW, int CH>
__global__ void __launch_bounds__(kTX * kTY) k_prep(PrepArgs a)
{
    __shared__ __align__(16) uint8_t gs[kTY + kMaxCH - 1][kGW];
    const int img = blockIdx.z;
    const uint32_t *__restrict__ rgbx = img ? a.rgbx[1] : a.rgbx[0];
    const uint8_t *__restrict__ grey = img ? a.grey[1] : a.grey[0];
    const int W = a.W, H = a.H;
    const int cw = CW ? CW : a.cw, ch = CH ? CH : a.ch;
    const int rx = cw / 2, ry = ch / 2;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    for (int r = threadIdx.y; r < kTY + 2 * ry; r += kTY) {
        const int y = min(max(y0 - ry + r, 0), H - 1);
        for (int c = threadIdx.x; c < kTX + 2 * rx; c += kTX) {
            const int x = min(max(x0 - rx + c, 0), W - 1);
            gs[r][c] = __ldg(grey + (size_t)y * W + x);
        }
    }
    __syncthreads();
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x = x0 + tx, y = y0 + ty;
    if (x >= W || y >= H) return;

    // census: bit k = [Y(n) < Y(p)], window row-major, centre skipped
    const uint32_t yc = gs[ty + ry][tx + rx];
    unsigned long long bits = 0ull;
    if (CW == 9 && CH == 7) {
        const uint32_t c4 = yc * 0x01010101u;
        const int al = tx & ~3, sh = 8 * (tx & 3);
        int k = 0;
#pragma unroll
        for (int dy = 0; dy < 7; dy++) {
            const uint32_t *row = reinterpret_cast<const uint32_t *>(&gs[ty + dy][al]);
            const uint32_t a0 = row[0], a1 = row[1], a2 = row[2];
            const uint32_t w0 = __funnelshift_r(a0, a1, sh);   // bytes dx 0..3
            const uint32_t w1 = __funnelshift_r(a1, a2, sh);   // bytes dx 4..7
            const uint32_t b8 = (__funnelshift_r(a2, 0u, sh) & 0xffu) < yc ? 1u : 0u;   // dx 8
            const uint32_t f0 = lt4(w0, c4), f1 = lt4(w1, c4);
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
    const uint32_t p = __ldg(rgbx + i);
    const int L1 = a.L1, L2 = a.L2;
    // a threshold >= 256 never stops an arm (channel differences are <= 255)
    const bool use1 = a.tau1 < 256, use2 = a.tau2 < 256;
    const uint32_t t1 = 0x01010101u * (uint32_t)min(a.tau1, 255);
    const uint32_t t2 = 0x01010101u * (uint32_t)min(a.tau2, 255);
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
        uint32_t prev = p;
        int n = 0;
        bool open = true;
#pragma unroll
        for (int u = 0; u < kArmBatch; u++) {
            const int j = u + 1;
            if (open && j <= lim[e]) {
                const uint32_t c = cand[e][u];
                if ((use1 && (any_ge(c, p, t1) || any_ge(c, prev, t1))) || (j > L2 && use2 && any_ge(c, p, t2)))
                    open = false;
                else {
                    n = j;
                    prev = c;
                }
            } else {
                open = false;
            }
        }
        // rare long arms: continue one candidate at a time
        for (int j = kArmBatch + 1; open && j <= lim[e]; j++) {
            const uint32_t c = __ldg(rgbx + i + j * step[e]);
            if ((use1 && (any_ge(c, p, t1) || any_ge(c, prev, t1))) || (j > L2 && use2 && any_ge(c, p, t2)))
                break;
            n = j;
            prev = c;
        }
        arm[e] = n;
    }
    const int lmin = min(min(arm[0], arm[1]), min(arm[2], arm[3]));
    const float alphaS = __ldg(a.tables + kTabAD + kTabCen + lmin);
    (img ? a.rec[1] : a.rec[0])[(size_t)y * a.rpitch + x] =
        make_uint4((uint32_t)bits, (uint32_t)(bits >> 32), p | (uint32_t(lmin) << 24), __float_as_uint(alphaS));
    (img ? a.arms[1] : a.arms[0])[i] = make_uchar4((uint8_t)arm[0], (uint8_t)arm[1], (uint8_t)arm[2], (uint8_t)arm[3]);
}

// ------------------------------------------------------------------ k_hagg
// Block = one row segment of one reference view for one group of 32
// disparities (lane = disparity d0 + 32*g + lane).  Stage 0 copies (cp.async)
// the tables, the reference records of the prefix range [xa, xb) (the
// output columns plus an L1 reach on both sides), the candidate records of
// the group and the output columns' arms into shared memory.  Then:
//   A. each warp walks a segment of kHSeg columns: Eq. 1 cost rounded to
//      fixed point, local inclusive prefix into P[x - xa][lane];
//   B. segment totals -> exclusive offsets, added to P in place;
//   C. every output column xo: S_H = P(xo + r) - P(xo - l - 1) (the
//      horizontal part of Eq. 2).
// Unsigned wrap-around makes the P differences exact segment sums.
constexpr int kTabBytes = (kTabAD + kTabCen) * 4;
constexpr int kHU = 4;

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
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// byte offsets of the H block's shared-memory regions
struct HSmem {
    int ref, oth, arm, p, t, total;
    __host__ __device__ HSmem(int len, int chunk, int nw)
    {
        ref = kTabBytes;
        oth = ref + len * 16;
        arm = oth + (len + 32) * 16;
        p = arm + (chunk + 3) / 4 * 16;
        t = p + len * 128;
        total = t + nw * 128;
    }
};

__global__ void __launch_bounds__(16 * 32) k_hagg(HArgs a)
{
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int W = a.W, L1 = a.L1;
    const int y = blockIdx.y;
    const int view = blockIdx.z / a.ngroups, g = blockIdx.z % a.ngroups;
    const int xs = blockIdx.x * a.chunk, xe = min(W, xs + a.chunk);
    const int xa = max(0, xs - L1), xb = min(W, xe + L1), len = xb - xa;
    const HSmem L(len, a.chunk, nw);
    float *sTA = reinterpret_cast<float *>(smem_raw);
    float *sTC = sTA + kTabAD;
    uint4 *sref = reinterpret_cast<uint4 *>(smem_raw + L.ref);
    uint4 *soth = reinterpret_cast<uint4 *>(smem_raw + L.oth);
    uchar4 *sarm = reinterpret_cast<uchar4 *>(smem_raw + L.arm);
    uint32_t *P = reinterpret_cast<uint32_t *>(smem_raw + L.p);   // [len][32]
    uint32_t *T = reinterpret_cast<uint32_t *>(smem_raw + L.t);   // [nw][32]

    // disparities of this group: [dlo, dhi] live
    const int dlo = a.d0 + 32 * g;
    const int dhi = min(min(a.d0 + a.dc, a.D), dlo + 32) - 1;
    const int sign = view ? 1 : -1;
    const int olo = view ? xa + dlo : xa - dhi;                 // candidate range [olo, olo + len + dhi - dlo)
    const int olen = len + dhi - dlo;
    const uint4 *rref = (view ? a.rec[1] : a.rec[0]) + (size_t)y * a.rpitch;
    const uint4 *roth = (view ? a.rec[0] : a.rec[1]) + (size_t)y * a.rpitch;   // padded: olo >= -255
    const uchar4 *aref = (view ? a.arms[1] : a.arms[0]) + (size_t)y * W;

    // ---- 0: stage
    for (int i = threadIdx.x; i < kTabBytes / 16; i += blockDim.x)
        cp_async16(smem_raw + 16 * i, reinterpret_cast<const uint8_t *>(a.tables) + 16 * i);
    for (int i = threadIdx.x; i < len; i += blockDim.x) cp_async16(sref + i, rref + xa + i);
    for (int i = threadIdx.x; i < olen; i += blockDim.x) cp_async16(soth + i, roth + olo + i);
    for (int i = threadIdx.x; i < xe - xs; i += blockDim.x) cp_async4(sarm + i, aref + xs + i);
    cp_async_wait_all();
    __syncthreads();

    const int d = dlo + lane;
    const bool live = d <= dhi;
    const int oi = (live ? sign * d : sign * dlo) - olo;   // candidate index = x + oi (in range)
    // columns x (relative to xa) whose match x -/+ d lies in the image
    const int vlo = live ? (view ? 0 : max(0, d - xa)) : 1, vhi = live ? (view ? W - d - xa : len) : 0;
    const float Sf = a.S;
    const uint32_t Sint = a.Sint;

    // ---- A: costs and local prefix of this warp's segment
    const int sa = warp * kHSeg, sb = min(len, sa + kHSeg);   // relative to xa
    uint32_t run = 0;
    auto cost_at = [&](const uint4 pr, const uint4 po, int x) -> uint32_t {
        const int h = __popc(pr.x ^ po.x) + __popc(pr.y ^ po.y);
        const int k = (int)__dp4a(__vabsdiffu4(pr.z, po.z), 0x00010101u, 0u);
        const float av = __uint_as_float(pr.w);
        const uint32_t q = __float2uint_rn(fmaf(av, sTA[k], (Sf - av) * sTC[h]));
        return (unsigned)(x - vlo) < (unsigned)(vhi - vlo) ? q : Sint;   // match outside the image: cost 1
    };
    int x0 = sa;
    for (; x0 + kHU <= sb; x0 += kHU) {
        uint4 pr[kHU], po[kHU];
#pragma unroll
        for (int u = 0; u < kHU; u++) {
            pr[u] = sref[x0 + u];
            po[u] = soth[x0 + u + xa + oi];
        }
        uint32_t c[kHU];
#pragma unroll
        for (int u = 0; u < kHU; u++) c[u] = cost_at(pr[u], po[u], x0 + u);
#pragma unroll
        for (int u = 0; u < kHU; u++) {
            run += c[u];
            P[(x0 + u) * 32 + lane] = run;
        }
    }
    for (; x0 < sb; x0++) {
        run += cost_at(sref[x0], soth[x0 + xa + oi], x0);
        P[x0 * 32 + lane] = run;
    }
    T[warp * 32 + lane] = run;
    __syncthreads();
    // ---- B: exclusive segment offsets, added in place
    uint32_t offs = 0;
    for (int w = 0; w < warp; w++) offs += T[w * 32 + lane];
    if (warp > 0) {
        uint32_t *q = P + sa * 32 + lane;
        int x = sa;
        for (; x + 8 <= sb; x += 8) {
#pragma unroll
            for (int u = 0; u < 8; u++) q[u * 32] += offs;
            q += 256;
        }
        for (; x < sb; x++, q += 32) *q += offs;
    }
    __syncthreads();
    // ---- C: horizontal segment sums of the output columns
    const int n_out = xe - xs, base = xs - xa;
    const size_t ostep = (size_t)nw * a.dstride;
    uint32_t *o = (view ? a.sh[1] : a.sh[0]) + ((size_t)y * W + xs + warp) * a.dstride + g * 32 + lane;
    const uint32_t *Pl = P + lane;
    int i = warp;
    for (; i + nw < n_out; i += 2 * nw, o += 2 * ostep) {
        const uchar4 am0 = sarm[i], am1 = sarm[i + nw];
        const int hi0 = base + i + am0.y, lo0 = base + i - am0.x - 1;   // lo >= -1
        const int hi1 = base + i + nw + am1.y, lo1 = base + i + nw - am1.x - 1;
        const uint32_t v0 = Pl[hi0 * 32] - (lo0 >= 0 ? Pl[lo0 * 32] : 0u);
        const uint32_t v1 = Pl[hi1 * 32] - (lo1 >= 0 ? Pl[lo1 * 32] : 0u);
        o[0] = v0;
        o[ostep] = v1;
    }
    if (i < n_out) {
        const uchar4 am = sarm[i];
        const int hi = base + i + am.y, lo = base + i - am.x - 1;
        *o = Pl[hi * 32] - (lo >= 0 ? Pl[lo * 32] : 0u);
    }
}

// ------------------------------------------------------------------ k_vagg
// Block = one column x of one reference view, a chunk of output rows.  The
// prefix range [ya, yb) is split into warp segments of 32 rows.  For each
// group of 32 disparities of the pass:
//   A. lane = disparity: each warp loads its 32 slice rows into registers
//      (one 128-byte line per row), sums them, exchanges the segment sums
//      with the other warps, and writes the column prefix (with its segment
//      offset) to Q[y - ya][lane] (row stride 33 words): one shared store per
//      evaluation;
//   C. lane = output row: V(d) = Q(y + dn, d) - Q(y - up - 1, d) for the 32
//      disparities (Eq. 2: the sum over the vertical arm of the horizontal
//      sums; N does not depend on d, so the WTA compares V), running minimum
//      with the smallest d on ties (Eq. 3) in registers across groups.
// Finally the running best is merged with earlier passes and written.
constexpr int kQS = 33;   // Q row stride: column d of consecutive rows hits distinct banks
constexpr int kVSeg = 32; // rows per warp

__host__ __device__ inline size_t vagg_smem_words(int len, int nw) { return (size_t)len * kQS + nw * 32 + 2 * len + nw; }

__global__ void __launch_bounds__(16 * 32, 2) k_vagg(VArgs a)
{
    extern __shared__ __align__(16) uint32_t vsmem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int W = a.W, H = a.H, L1 = a.L1;
    const int x = blockIdx.x, view = blockIdx.y;
    const int ys = blockIdx.z * a.chunk, ye = min(H, ys + a.chunk);
    const int ya = max(0, ys - L1), yb = min(H, ye + L1);
    const int len = yb - ya;
    uint32_t *Q = vsmem;                      // [len][kQS]
    uint32_t *T = Q + len * kQS;              // [nw][32] segment sums
    uint32_t *NQ = T + nw * 32;               // [len] prefix of l + r + 1
    uint32_t *NT = NQ + len;                  // [nw]
    uint32_t *AW = NT + nw;                   // [len] arm words

    const uint32_t *sh = (view ? a.sh[1] : a.sh[0]) + (size_t)x * a.dstride + lane;
    const uint32_t *arms = reinterpret_cast<const uint32_t *>(view ? a.arms[1] : a.arms[0]) + x;
    const size_t rowstride = (size_t)W * a.dstride;
    const int sa = warp * kVSeg, sb = min(len, sa + kVSeg);   // relative to ya
    const int ng = (a.dc + 31) / 32;
    const bool want_vol = a.vol != nullptr && view == a.vol_view;

    // arm word of this lane's row and the region-size prefix (d independent)
    const int r = sa + lane;
    const bool rin = r < sb;
    const uint32_t aw = rin ? __ldg(arms + (size_t)(ya + r) * W) : 0u;
    {
        uint32_t nv = rin ? (aw & 0xffu) + ((aw >> 8) & 0xffu) + 1u : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {   // inclusive scan across the segment's rows
            const uint32_t t = __shfl_up_sync(0xffffffffu, nv, o);
            if (lane >= o) nv += t;
        }
        if (rin) { AW[r] = aw; NQ[r] = nv; }
        if (lane == 31) NT[warp] = nv;
    }
    const bool out_row = rin && ya + r >= ys && ya + r < ye;
    uint32_t bv = 0xffffffffu, bd = 0;

    for (int g = 0; g < ng; g++) {
        // ---- A: this warp's 32 rows of the slice column, lane = disparity
        uint32_t v[kVSeg];
        const uint32_t *src = sh + (size_t)(ya + sa) * rowstride + g * 32;
#pragma unroll
        for (int u = 0; u < kVSeg; u++) v[u] = sa + u < sb ? __ldg(src + (size_t)u * rowstride) : 0u;
        uint32_t tot = 0;
#pragma unroll
        for (int u = 0; u < kVSeg; u++) tot += v[u];
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
        uint32_t *q = Q + sa * kQS + lane;
#pragma unroll
        for (int u = 0; u < kVSeg; u++) {
            run += v[u];
            if (sa + u < sb) q[u * kQS] = run;
        }
        __syncthreads();
        // ---- C: lane = output row, loop over the group's disparities
        const int dbase = a.d0 + g * 32;
        const int nlive = max(0, min(32, min(a.dc - g * 32, a.D - dbase)));
        if (out_row) {
            const int up = (aw >> 16) & 0xff, dn = aw >> 24;
            const uint32_t *qh = Q + (r + dn) * kQS;
            const int lo = r - up - 1;
            const uint32_t *ql = Q + max(lo, 0) * kQS;
            const uint32_t lomask = lo >= 0 ? 0xffffffffu : 0u;
#pragma unroll 8
            for (int j = 0; j < 32; j++) {
                const uint32_t vv = qh[j] - (ql[j] & lomask);
                if (j < nlive && vv < bv) { bv = vv; bd = (uint32_t)(dbase + j); }
            }
            if (want_vol) {
                const uint32_t n = NQ[r + dn] - (lo >= 0 ? NQ[lo] : 0u);
                for (int j = 0; j < nlive; j++) {
                    const uint32_t vv = qh[j] - (ql[j] & lomask);
                    a.vol[((size_t)(dbase + j) * H + ya + r) * W + x] = float(vv) / (float(n) * a.S);
                }
            }
        }
        __syncthreads();   // Q and T are reused by the next group
    }
    // ---- merge with earlier passes, write the disparity (last pass) or state
    if (!out_row) return;
    unsigned long long *best = view ? a.best[1] : a.best[0];
    int16_t *disp = view ? a.disp[1] : a.disp[0];
    float *cost = view ? a.cost[1] : a.cost[0];
    const size_t i = (size_t)(ya + r) * W + x;
    unsigned long long key = ((unsigned long long)bv << 32) | bd;
    if (!a.first) {
        const unsigned long long prev = best[i];
        key = prev <= key ? prev : key;   // earlier passes hold smaller d
    }
    if (a.last) {
        disp[i] = (int16_t)(key & 0xffffffffu);
        if (cost) {
            const int up = (aw >> 16) & 0xff, dn = aw >> 24;
            const int lo = r - up - 1;
            const uint32_t n = NQ[r + dn] - (lo >= 0 ? NQ[lo] : 0u);
            cost[i] = float(uint32_t(key >> 32)) / (float(n) * a.S);
        }
    } else {
        best[i] = key;
    }
}

// ------------------------------------------------------------------ k_lr
__global__ void k_lr(const int16_t *__restrict__ dl, const int16_t *__restrict__ dr, int W, int H,
                     int tol, int16_t *__restrict__ out)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)W * H) return;
    const int x = int(i % W);
    const int d = dl[i];
    int16_t r = -1;
    if (tol < 0) r = (int16_t)d;
    else if (d >= 0 && x - d >= 0) {
        const int d2 = dr[i - d];
        if (d2 >= 0 && abs(d - d2) <= tol) r = (int16_t)d;
    }
    out[i] = r;
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
};

struct Layout {
    size_t rgbx[2], grey[2], rec[2], arms[2], best[2], disp[2], sh[2], total;
    int dc, dstride, npass, rpitch;
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
    return true;
}

bool params_valid(const dco_params &p)
{
    if (!(p.lambda_ad > 0.f) || !(p.lambda_census > 0.f) || !(p.eps > 0.f) || !(p.gamma_l >= 0.f))
        return false;
    if (p.census_w < 1 || p.census_h < 1 || !(p.census_w & 1) || !(p.census_h & 1)) return false;
    if (p.census_w > kMaxCW || p.census_h > kMaxCH || p.census_w * p.census_h - 1 > 64) return false;
    if (p.arm_l1 < 1 || p.arm_l1 > kMaxL1 || p.arm_l2 < 0 || p.tau1 < 0 || p.tau2 < 0) return false;
    if (p.d_chunk < 0) return false;
    return true;
}

bool dims_valid(int W, int H, int D)
{
    return W >= 1 && H >= 1 && W <= 16384 && H <= 16384 && D >= 1 && D <= 256 && D <= W;
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
    for (int v = 0; v < 2; v++) { L.rgbx[v] = off; off = align_up(off + 4 * npx); }
    for (int v = 0; v < 2; v++) { L.grey[v] = off; off = align_up(off + npx); }
    for (int v = 0; v < 2; v++) { L.rec[v] = off; off = align_up(off + 16 * (size_t)H * L.rpitch); }
    for (int v = 0; v < 2; v++) { L.arms[v] = off; off = align_up(off + 4 * npx); }
    for (int v = 0; v < 2; v++) { L.best[v] = off; off = align_up(off + (L.npass > 1 ? 8 * npx : 0)); }
    for (int v = 0; v < 2; v++) { L.disp[v] = off; off = align_up(off + 2 * npx); }
    for (int v = 0; v < 2; v++) { L.sh[v] = off; off = align_up(off + 4 * npx * (size_t)L.dstride); }
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

HGeom hagg_geom(int W, int H, int dc, int L1)
{
    HGeom g{};
    g.chunk = W <= kHMaxLen ? W : 512;
    const int len = std::min(W, g.chunk + 2 * L1);
    g.nw = (len + kHSeg - 1) / kHSeg;
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

VGeom vagg_geom(int W, int H, int L1)
{
    VGeom g{};
    // at most 16 warps of 32 rows: the prefix range (chunk + 2*L1) <= 512
    const int nchunks = H <= 512 ? 1 : (H + (512 - 2 * kMaxL1) - 1) / (512 - 2 * kMaxL1);
    g.chunk = (H + nchunks - 1) / nchunks;
    const int len = std::min(H, g.chunk + 2 * L1);
    g.seglog = 5;   // 32 rows per warp, one output row per lane
    g.nw = (len + kVSeg - 1) / kVSeg;
    g.smem = vagg_smem_words(len, g.nw) * 4;
    g.grid = dim3(W, 2, nchunks);
    return g;
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
    unsigned long long launches = 0;
    std::vector<ProfEvent> pending;
    std::vector<cudaEvent_t> pool;
    std::vector<ProfAgg> agg;
    std::string last_error;
};

namespace {

dco_status cuda_fail(dco_stereo *h, cudaError_t e, const char *what)
{
    if (h) h->last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? DCO_ENOMEM : DCO_ECUDA;
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
    ProfScope(dco_stereo *h_, cudaStream_t s_, const char *name) : h(h_), s(s_)
    {
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
        if (h->profiling) {
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

dco_status ensure_tables(dco_stereo *h, const dco_params &p, const Derived &dv, cudaStream_t s)
{
    const float key[4] = {p.lambda_ad, p.lambda_census, p.gamma_l, p.eps};
    if (h->tab_valid && !std::memcmp(key, h->tab_key, sizeof key) && h->tab_l1 == p.arm_l1) return DCO_OK;
    float *t = h->h_tables;
    // Eq. 1 terms, evaluated in double on the host and rounded once to float
    for (int k = 0; k < kTabAD; k++)
        t[k] = k <= 765 ? (float)(1.0 - std::exp(-(k / 3.0) / (double)p.lambda_ad)) : 1.0f;
    for (int k = 0; k < kTabCen; k++)
        t[kTabAD + k] = k <= 64 ? (float)(1.0 - std::exp(-(double)k / (double)p.lambda_census)) : 1.0f;
    for (int l = 0; l < kTabAlpha; l++) {
        const double alpha = 1.0 - std::exp(-(double)p.gamma_l / ((double)l + (double)p.eps));
        t[kTabAD + kTabCen + l] = (float)(alpha * (double)dv.Sint);
    }
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

// first real record of row 0 of a padded record array
uint4 *rec_ptr(dco_stereo *h, size_t off) { return ws_ptr<uint4>(h, off) + kRPad; }

// grey/colour packing and census + arms for nimg images (1 or 2); arms of
// image 0 go to arms0 (the caller's buffer for the arms entry point)
dco_status launch_prep(dco_stereo *h, const dco_params &p, const Derived &dv, const Layout &L,
                       const uint8_t *img0, const uint8_t *img1, int nimg, uchar4 *arms0, int W, int H,
                       cudaStream_t s)
{
    const int npx = W * H;
    {
        PackArgs a{};
        a.rgb[0] = img0; a.rgb[1] = img1;
        for (int v = 0; v < 2; v++) {
            a.rgbx[v] = ws_ptr<uint32_t>(h, L.rgbx[v]);
            a.grey[v] = ws_ptr<uint8_t>(h, L.grey[v]);
        }
        a.npx = npx;
        ProfScope ps(h, s, "k_pack");
        k_pack<<<dim3((npx / 4 + 256) / 256, nimg), 256, 0, s>>>(a);
        DCO_CUDA(h, cudaGetLastError());
    }
    PrepArgs a{};
    for (int v = 0; v < 2; v++) {
        a.rgbx[v] = ws_ptr<uint32_t>(h, L.rgbx[v]);
        a.grey[v] = ws_ptr<uint8_t>(h, L.grey[v]);
        a.rec[v] = rec_ptr(h, L.rec[v]);
        a.arms[v] = ws_ptr<uchar4>(h, L.arms[v]);
    }
    if (arms0) a.arms[0] = arms0;
    a.tables = h->d_tables;
    a.W = W; a.H = H; a.rpitch = L.rpitch;
    a.cw = p.census_w; a.ch = p.census_h;
    a.L1 = dv.L1; a.L2 = p.arm_l2; a.tau1 = p.tau1; a.tau2 = p.tau2;
    dim3 grid((W + kTX - 1) / kTX, (H + kTY - 1) / kTY, nimg);
    ProfScope ps(h, s, "k_prep");
    if (p.census_w == 9 && p.census_h == 7) k_prep<9, 7><<<grid, dim3(kTX, kTY), 0, s>>>(a);
    else k_prep<0, 0><<<grid, dim3(kTX, kTY), 0, s>>>(a);
    DCO_CUDA(h, cudaGetLastError());
    return DCO_OK;
}

dco_status launch_pass(dco_stereo *h, const Layout &L, const Derived &dv, int W, int H, int D, int d0,
                       bool first, bool last, int16_t *disp_l, int16_t *disp_r, float *cost_l,
                       float *cost_r, float *vol, int vol_view, cudaStream_t s)
{
    const int dc = std::min(L.dc, D - d0);
    HArgs ha{};
    for (int v = 0; v < 2; v++) {
        ha.rec[v] = rec_ptr(h, L.rec[v]);
        ha.arms[v] = ws_ptr<uchar4>(h, L.arms[v]);
        ha.sh[v] = ws_ptr<uint32_t>(h, L.sh[v]);
    }
    ha.tables = h->d_tables;
    ha.W = W; ha.H = H; ha.D = D; ha.rpitch = L.rpitch;
    ha.d0 = d0; ha.dc = dc; ha.dstride = L.dstride;
    ha.ngroups = (dc + 31) / 32;
    ha.L1 = dv.L1; ha.S = dv.S; ha.Sint = dv.Sint;
    {
        const HGeom g = hagg_geom(W, H, dc, dv.L1);
        ha.chunk = g.chunk;
        ProfScope ps(h, s, "k_hagg");
        cudaFuncSetAttribute(k_hagg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
        k_hagg<<<g.grid, g.nw * 32, g.smem, s>>>(ha);
        DCO_CUDA(h, cudaGetLastError());
    }
    VArgs va{};
    for (int v = 0; v < 2; v++) {
        va.sh[v] = ha.sh[v];
        va.arms[v] = ha.arms[v];
        va.best[v] = ws_ptr<unsigned long long>(h, L.best[v]);
    }
    va.disp[0] = disp_l; va.disp[1] = disp_r;
    va.cost[0] = cost_l; va.cost[1] = cost_r;
    va.vol = vol; va.vol_view = vol_view;
    va.W = W; va.H = H; va.D = D; va.d0 = d0; va.dc = dc; va.dstride = L.dstride;
    va.first = first; va.last = last;
    va.L1 = dv.L1; va.S = dv.S;
    {
        const VGeom g = vagg_geom(W, H, dv.L1);
        va.chunk = g.chunk;
        va.seglog = g.seglog;
        ProfScope ps(h, s, "k_vagg");
        cudaFuncSetAttribute(k_vagg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
        k_vagg<<<g.grid, g.nw * 32, g.smem, s>>>(va);
        DCO_CUDA(h, cudaGetLastError());
    }
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
    DCO_CUDA(h, cudaSetDevice(h->device));
    return DCO_OK;
}

dco_status run_match(dco_stereo *h, const uint8_t *left, const uint8_t *right, int W, int H, int D,
                     const dco_params &p, int16_t *disp_out, int16_t *disp_l, int16_t *disp_r,
                     float *cost_l, float *cost_r, float *vol, int vol_view, cudaStream_t s)
{
    Derived dv;
    derive(p, dv);
    Layout L = make_layout(W, H, D, p);
    if (h->budget && L.total > h->budget) {
        // shrink the pass until the slices fit
        for (int dc = (L.dc / 32) * 32; dc >= 32; dc -= 32) {
            Layout L2 = make_layout(W, H, D, p, dc);
            if (L2.total <= h->budget) { L = L2; break; }
        }
    }
    dco_status st = ensure_ws(h, L.total);
    if (st != DCO_OK) return st;
    if ((st = ensure_tables(h, p, dv, s)) != DCO_OK) return st;
    if (!disp_l) disp_l = ws_ptr<int16_t>(h, L.disp[0]);
    if (!disp_r) disp_r = ws_ptr<int16_t>(h, L.disp[1]);
    if ((st = launch_prep(h, p, dv, L, left, right, 2, nullptr, W, H, s)) != DCO_OK)
        return st;
    for (int d0 = 0; d0 < D; d0 += L.dc) {
        const bool first = d0 == 0, last = d0 + L.dc >= D;
        if ((st = launch_pass(h, L, dv, W, H, D, d0, first, last, disp_l, disp_r, cost_l, cost_r, vol,
                              vol_view, s)) != DCO_OK)
            return st;
    }
    if (disp_out) {
        const size_t n = (size_t)W * H;
        ProfScope ps(h, s, "k_lr");
        k_lr<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(disp_l, disp_r, W, H, p.lr_tol, disp_out);
        DCO_CUDA(h, cudaGetLastError());
    }
    return DCO_OK;
}

} // namespace

// ===================================================================== C ABI
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
    delete h;
}

size_t dco_stereo_workspace_bytes(int W, int H, int D, const dco_params *pin)
{
    dco_params p;
    if (pin) p = *pin;
    else dco_params_default(&p);
    if (!params_valid(p) || !dims_valid(W, H, D)) return 0;
    return make_layout(W, H, D, p).total;
}

dco_status dco_stereo_reserve(dco_stereo *h, int W, int H, int D, const dco_params *pin)
{
    dco_params p;
    dco_status st = check_common(h, pin, p);
    if (st != DCO_OK) return st;
    if (!dims_valid(W, H, D)) return DCO_EINVAL;
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
    if (!left || !right || !dims_valid(W, H, D)) return DCO_EINVAL;
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

dco_status dco_stereo_match_host(dco_stereo *h, const uint8_t *left_host, const uint8_t *right_host, int W,
                                 int H, int D, const dco_params *pin, int16_t *disp_host, dco_stream stream)
{
    dco_params p;
    dco_status st = check_common(h, pin, p);
    if (st != DCO_OK) return st;
    if (!left_host || !right_host || !disp_host || !dims_valid(W, H, D)) return DCO_EINVAL;
    const size_t img = (size_t)W * H * 3, out = (size_t)W * H * 2;
    const size_t need = align_up(img) * 2 + align_up(out);
    cudaStream_t s = (cudaStream_t)stream;
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

dco_status dco_stereo_census(dco_stereo *h, const uint8_t *rgb, int W, int H, const dco_params *pin,
                             uint64_t *census_out, dco_stream stream)
{
    dco_params p;
    dco_status st = check_common(h, pin, p);
    if (st != DCO_OK) return st;
    if (!rgb || !census_out || !dims_valid(W, H, 1)) return DCO_EINVAL;
    Derived dv;
    derive(p, dv);
    Layout L = make_layout(W, H, 1, p);
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_ws(h, L.total)) != DCO_OK) return st;
    if ((st = ensure_tables(h, p, dv, s)) != DCO_OK) return st;
    if ((st = launch_prep(h, p, dv, L, rgb, rgb, 1, nullptr, W, H, s)) != DCO_OK)
        return st;
    const size_t n = (size_t)W * H;
    ProfScope ps(h, s, "k_extract_census");
    k_extract_census<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rec_ptr(h, L.rec[0]), W, H, L.rpitch,
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
    Derived dv;
    derive(p, dv);
    Layout L = make_layout(W, H, 1, p);
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_ws(h, L.total)) != DCO_OK) return st;
    if ((st = ensure_tables(h, p, dv, s)) != DCO_OK) return st;
    if ((st = launch_prep(h, p, dv, L, rgb, rgb, 1, reinterpret_cast<uchar4 *>(arms_out), W, H, s)) != DCO_OK)
        return st;
    return DCO_OK;
}

dco_status dco_stereo_cost_volume(dco_stereo *h, const uint8_t *left, const uint8_t *right, int W, int H,
                                  int D, const dco_params *pin, int view, float *vol_out, dco_stream stream)
{
    dco_params p;
    dco_status st = check_common(h, pin, p);
    if (st != DCO_OK) return st;
    if (!left || !right || !vol_out || (view != 0 && view != 1) || !dims_valid(W, H, D)) return DCO_EINVAL;
    return run_match(h, left, right, W, H, D, p, nullptr, nullptr, nullptr, nullptr, nullptr, vol_out, view,
                     (cudaStream_t)stream);
}

dco_status dco_stereo_lr_check(dco_stereo *h, const int16_t *dl, const int16_t *dr, int W, int H, int tol,
                               int16_t *out, dco_stream stream)
{
    if (!h || !dl || !dr || !out || W < 1 || H < 1) return DCO_EINVAL;
    DCO_CUDA(h, cudaSetDevice(h->device));
    const size_t n = (size_t)W * H;
    cudaStream_t s = (cudaStream_t)stream;
    ProfScope ps(h, s, "k_lr");
    k_lr<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dl, dr, W, H, tol, out);
    DCO_CUDA(h, cudaGetLastError());
    return DCO_OK;
}

dco_status dco_stereo_match_batch(dco_stereo *h, const dco_pair_desc *descs, int n, const dco_params *pin,
                                  dco_stream stream)
{
    dco_params p;
    dco_status st = check_common(h, pin, p);
    if (st != DCO_OK) return st;
    if (n < 0 || (n > 0 && !descs)) return DCO_EINVAL;
    for (int i = 0; i < n; i++)
        if (!descs[i].left || !descs[i].right || !descs[i].disp_out ||
            !dims_valid(descs[i].W, descs[i].H, descs[i].D))
            return DCO_EINVAL;
    for (int i = 0; i < n; i++) {
        st = run_match(h, descs[i].left, descs[i].right, descs[i].W, descs[i].H, descs[i].D, p,
                       descs[i].disp_out, nullptr, nullptr, nullptr, nullptr, nullptr, 0, (cudaStream_t)stream);
        if (st != DCO_OK) return st;
    }
    return DCO_OK;
}

dco_status dco_stereo_sync_status(dco_stereo *h)
{
    if (!h) return DCO_EINVAL;
    DCO_CUDA(h, cudaSetDevice(h->device));
    DCO_CUDA(h, cudaDeviceSynchronize());
    int v = 0;
    DCO_CUDA(h, cudaMemcpy(&v, h->d_status, sizeof v, cudaMemcpyDeviceToHost));
    DCO_CUDA(h, cudaMemset(h->d_status, 0, sizeof v));
    return v ? DCO_EDEVICE : DCO_OK;
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
std::mutex g_noalloc_mu;
void *g_noalloc_base[kNoAllocMaxDevices] = {};
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
    if (!params_valid(p) || !left || !right || !disp_out || !dims_valid(W, H, D)) return DCO_EINVAL;
    p.d_chunk = 32;   // passes of 32 disparities keep the slices small
    Derived dv;
    derive(p, dv);
    const size_t tab_bytes = align_up(sizeof(float) * kTabFloats);
    const Layout L = make_layout(W, H, D, p);
    if (tab_bytes + L.total > kNoAllocScratchBytes) return DCO_EBUDGET;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DCO_ECUDA;
    void *base = nullptr;
    dco_status st = noalloc_base(dev, &base);
    if (st != DCO_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;

    // Eq. 1 tables (host double, rounded once to float) into the scratch
    float tab[kTabFloats];
    for (int k = 0; k < kTabAD; k++)
        tab[k] = k <= 765 ? (float)(1.0 - std::exp(-(k / 3.0) / (double)p.lambda_ad)) : 1.0f;
    for (int k = 0; k < kTabCen; k++)
        tab[kTabAD + k] = k <= 64 ? (float)(1.0 - std::exp(-(double)k / (double)p.lambda_census)) : 1.0f;
    for (int l = 0; l < kTabAlpha; l++) {
        const double alpha = 1.0 - std::exp(-(double)p.gamma_l / ((double)l + (double)p.eps));
        tab[kTabAD + kTabCen + l] = (float)(alpha * (double)dv.Sint);
    }
    if (cudaMemcpyAsync(base, tab, sizeof tab, cudaMemcpyHostToDevice, s) != cudaSuccess) return DCO_ECUDA;

    // a handle that owns nothing: its workspace and tables are the scratch
    dco_stereo view;
    view.device = dev;
    view.ws = static_cast<char *>(base) + tab_bytes;
    view.ws_cap = kNoAllocScratchBytes - tab_bytes;
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
    return st;
}
