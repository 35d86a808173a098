// Depth densification of Sect. 6 (Eqs. 13-20) on the GPU: the normal
// equations of the Eq. 20 energy,
//   (lambda_d w_sparse + lambda_s2 w_stable) D(p) + 2 lambda_s sum_q w_pq (D(p) - D(q))
//       = lambda_d w_sparse D_sparse(p) + lambda_s2 w_stable D_pre(p),
// a 5-point symmetric system (N4 cut at the border), solved by conjugate
// gradients with a Jacobi preconditioner, matrix free.  Included by
// dco_stereo.cu after the handle helpers.
//
// Per iteration two launches:
//   k_dn_ap   p_new = z + beta p_old (both buffers kept: neighbours read the
//             old one) and Ap = A p_new; alpha = r.z / p.Ap;
//   k_dn_upd  x += alpha p, r -= alpha Ap, z = r / diag; beta = r.z / previous r.z.
// Dot products: FP32 products and warp sums, double block sums written as
// block partials; the last block of the launch to finish (an atomic counter
// after a memory fence, no waiting) adds the partials in index order, so the
// scalars are deterministic, and updates them.  Every batch of iterations
// ends with a residual replacement (k_dn_resid: r = b - A x in double) and the
// convergence test on that true residual; once it is below tol, a device flag
// makes every later launch return at once.

namespace dco {

constexpr int kDnBlock = 256;

struct DnScalars {
    double rz, pap, rr, bb, alpha, beta;
    int done, iters;
    unsigned count;   // blocks of the current launch that have written their partials
};

struct DnArgs {
    const float *ds, *dpre, *mf, *mi;
    const uint8_t *contour;
    float *x, *r, *z, *p[2], *ap, *wr, *wd, *dg, *b;
    double *part;          // [nblk][2]
    DnScalars *sc;
    int W, H, nblk;
    float lambda_d, lambda_s, lambda_s2;
    double tol2;           // tol^2
};

// Eq. 16 (with Eq. 17's s = M_fuse * M_I)
__device__ __forceinline__ float dn_weight(int bp, int bq, float sp, float sq)
{
    return bp + bq == 1 ? 0.0f : fmaxf(1.0f - fminf(sp, sq), 0.0f);
}

__device__ __forceinline__ float dn_s(const DnArgs &a, size_t i)
{
    return (a.mf ? a.mf[i] : 0.0f) * (a.mi ? a.mi[i] : 0.0f);
}

__device__ __forceinline__ int dn_b(const DnArgs &a, size_t i) { return a.contour ? (a.contour[i] != 0) : 0; }

// Block sums of (v0, v1) into part[blockIdx.x]; returns true in thread 0 of
// the last block to finish, with the sums over all blocks in t0, t1 (added in
// block order).  Every thread of every block must call it.
__device__ __forceinline__ bool dn_reduce(float v0, float v1, const DnArgs &a, double &t0, double &t1)
{
    __shared__ double s0[kDnBlock / 32], s1[kDnBlock / 32];
    __shared__ bool last;
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_down_sync(0xffffffffu, v0, o);
        v1 += __shfl_down_sync(0xffffffffu, v1, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { s0[w] = v0; s1[w] = v1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double u0 = 0.0, u1 = 0.0;
        for (int k = 0; k < kDnBlock / 32; k++) { u0 += s0[k]; u1 += s1[k]; }
        a.part[2 * blockIdx.x] = u0;
        a.part[2 * blockIdx.x + 1] = u1;
        __threadfence();
        last = atomicAdd(&a.sc->count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double u0 = 0.0, u1 = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
        u0 += __ldcg(a.part + 2 * k);
        u1 += __ldcg(a.part + 2 * k + 1);
    }
    for (int o = 16; o > 0; o >>= 1) {
        u0 += __shfl_down_sync(0xffffffffu, u0, o);
        u1 += __shfl_down_sync(0xffffffffu, u1, o);
    }
    __syncthreads();
    if (l == 0) { s0[w] = u0; s1[w] = u1; }
    __syncthreads();
    if (threadIdx.x != 0) return false;
    t0 = 0.0;
    t1 = 0.0;
    for (int k = 0; k < kDnBlock / 32; k++) { t0 += s0[k]; t1 += s1[k]; }
    a.sc->count = 0;   // for the next launch
    return true;
}

// weights, diagonal, right-hand side, initial guess (the data where present)
__global__ void __launch_bounds__(kDnBlock) k_dn_setup(const DnArgs a)
{
    const unsigned n = (unsigned)a.W * a.H, W = (unsigned)a.W;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.sc->count = 0;
        a.sc->done = 0;
    }
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned x = i % W, y = i / W;
        const int bp = dn_b(a, i);
        const float sp = dn_s(a, i);
        float sum = 0.0f, wr = 0.0f, wd = 0.0f;
        if (x > 0) sum += dn_weight(bp, dn_b(a, i - 1), sp, dn_s(a, i - 1));
        if (y > 0) sum += dn_weight(bp, dn_b(a, i - W), sp, dn_s(a, i - W));
        if (x + 1 < W) sum += (wr = dn_weight(bp, dn_b(a, i + 1), sp, dn_s(a, i + 1)));
        if (y + 1 < (unsigned)a.H) sum += (wd = dn_weight(bp, dn_b(a, i + W), sp, dn_s(a, i + W)));
        const float ds = a.ds[i], dp = a.dpre ? a.dpre[i] : 0.0f;
        const float wsp = ds > 0.0f ? a.lambda_d : 0.0f, wst = dp > 0.0f ? a.lambda_s2 : 0.0f;   // Eqs. 14, 19
        a.wr[i] = wr;
        a.wd[i] = wd;
        a.dg[i] = wsp + wst + 2.0f * a.lambda_s * sum;
        a.b[i] = wsp * ds + wst * dp;
        a.x[i] = ds > 0.0f ? ds : (dp > 0.0f ? dp : 0.0f);
        a.p[0][i] = 0.0f;
    }
}

// (A v)(i) = diag(i) v(i) - 2 lambda_s sum_q w_iq v(q)   (5-point stencil)
__device__ __forceinline__ float dn_apply(const DnArgs &a, const float *v, unsigned i, int x, int y)
{
    float nb = 0.0f;
    if (x + 1 < a.W) nb += a.wr[i] * v[i + 1];
    if (x > 0) nb += a.wr[i - 1] * v[i - 1];
    if (y + 1 < a.H) nb += a.wd[i] * v[i + a.W];
    if (y > 0) nb += a.wd[i - a.W] * v[i - a.W];
    return a.dg[i] * v[i] - 2.0f * a.lambda_s * nb;
}

// r = b - A x0, z = r / diag, partials of r.z and b.b
__global__ void __launch_bounds__(kDnBlock) k_dn_init(const DnArgs a)
{
    const unsigned n = (unsigned)a.W * a.H;
    float rz = 0.0f, bb = 0.0f;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int x = (int)(i % (unsigned)a.W), y = (int)(i / (unsigned)a.W);
        const float r = a.b[i] - dn_apply(a, a.x, i, x, y);
        const float d = a.dg[i];
        const float z = d > 0.0f ? r / d : 0.0f;
        a.r[i] = r;
        a.z[i] = z;
        rz += r * z;
        bb += a.b[i] * a.b[i];
    }
    double t0, t1;
    if (dn_reduce(rz, bb, a, t0, t1)) {
        DnScalars *sc = a.sc;
        sc->rz = t0;
        sc->bb = t1;
        sc->rr = t0;
        sc->beta = 0.0;
        sc->iters = 0;
        sc->done = !(t0 > 0.0) || !(t1 > 0.0);
    }
}

// p_new = z + beta p_old, Ap = A p_new (p_new of the neighbours formed on the fly)
__global__ void __launch_bounds__(kDnBlock) k_dn_ap(const DnArgs a, int it)
{
    if (a.sc->done) return;
    const unsigned n = (unsigned)a.W * a.H, W = (unsigned)a.W;
    const float *po = a.p[it & 1];
    float *pn = a.p[(it + 1) & 1];
    const float beta = (float)a.sc->beta;
    float pap = 0.0f;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned x = i % W, y = i / W;
        auto pv = [&](unsigned j) { return a.z[j] + beta * po[j]; };
        const float c = pv(i);
        float nb = 0.0f;
        if (x + 1 < W) nb += a.wr[i] * pv(i + 1);
        if (x > 0) nb += a.wr[i - 1] * pv(i - 1);
        if (y + 1 < (unsigned)a.H) nb += a.wd[i] * pv(i + W);
        if (y > 0) nb += a.wd[i - W] * pv(i - W);
        const float ap = a.dg[i] * c - 2.0f * a.lambda_s * nb;
        pn[i] = c;
        a.ap[i] = ap;
        pap += c * ap;
    }
    double t0, t1;
    if (dn_reduce(pap, 0.0f, a, t0, t1)) {
        a.sc->pap = t0;
        if (!(t0 > 0.0)) a.sc->done = 1;   // no direction left (solved, or breakdown)
        else a.sc->alpha = a.sc->rz / t0;
    }
}

// x += alpha p, r -= alpha Ap, z = r / diag; partials of r.z and r.r
__global__ void __launch_bounds__(kDnBlock) k_dn_upd(const DnArgs a, int it)
{
    if (a.sc->done) return;
    const unsigned n = (unsigned)a.W * a.H;
    const float alpha = (float)a.sc->alpha;
    const float *p = a.p[(it + 1) & 1];
    float rz = 0.0f, rr = 0.0f;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        a.x[i] += alpha * p[i];
        const float r = a.r[i] - alpha * a.ap[i];
        const float d = a.dg[i];
        const float z = d > 0.0f ? r / d : 0.0f;
        a.r[i] = r;
        a.z[i] = z;
        rz += r * z;
        rr += r * r;
    }
    double t0, t1;
    if (dn_reduce(rz, rr, a, t0, t1)) {
        DnScalars *sc = a.sc;
        sc->beta = sc->rz > 0.0 ? t0 / sc->rz : 0.0;
        sc->rz = t0;
        sc->rr = t1;
        sc->iters += 1;
        if (!(t0 > 0.0)) sc->done = 1;   // r = 0: solved
    }
}

// residual replacement: r = b - A x evaluated in double (the FP32 recursion
// drifts from the true residual), z = r / diag; partials of r.z and r.r
__global__ void __launch_bounds__(kDnBlock) k_dn_resid(const DnArgs a)
{
    if (a.sc->done) return;
    const unsigned n = (unsigned)a.W * a.H, W = (unsigned)a.W;
    float rz = 0.0f, rr = 0.0f;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned x = i % W, y = i / W;
        double nb = 0.0;
        if (x + 1 < W) nb += (double)a.wr[i] * a.x[i + 1];
        if (x > 0) nb += (double)a.wr[i - 1] * a.x[i - 1];
        if (y + 1 < (unsigned)a.H) nb += (double)a.wd[i] * a.x[i + W];
        if (y > 0) nb += (double)a.wd[i - W] * a.x[i - W];
        const double rd = (double)a.b[i] - ((double)a.dg[i] * a.x[i] - 2.0 * (double)a.lambda_s * nb);
        const float r = (float)rd, d = a.dg[i];
        const float z = d > 0.0f ? r / d : 0.0f;
        a.r[i] = r;
        a.z[i] = z;
        rz += r * z;
        rr += r * r;
    }
    double t0, t1;
    if (dn_reduce(rz, rr, a, t0, t1)) {
        DnScalars *sc = a.sc;
        sc->rz = t0;
        sc->rr = t1;
        if (t1 <= a.tol2 * sc->bb || !(t0 > 0.0)) sc->done = 1;
    }
}

}  // namespace dco
