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
    pdl_enter();
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
    pdl_enter();
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
    pdl_enter();
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
    pdl_enter();
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
    pdl_enter();
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

// ------------------------------------------------------------- C ABI
// (this header is included by dco_stereo.cu at file scope, after the handle
// and the launch helpers)
extern "C" {

dco_status dco_dense_params_default(dco_dense_params *p)
{
    if (!p) return DCO_EINVAL;
    p->lambda_d = 0.80f;    // Sect. 7.2
    p->lambda_s = 1.20f;
    p->lambda_s2 = 0.02f;
    p->tol = 1e-5f;
    p->max_iters = 4000;
    return DCO_OK;
}

dco_status dco_stereo_densify(dco_stereo *h, const float *d_sparse, const uint8_t *contour, const float *m_fuse,
                              const float *m_int, const float *d_pre, int W, int H, const dco_dense_params *pin,
                              float *d_out, dco_stream stream)
{
    if (!h || !d_sparse || !d_out || W < 1 || H < 1 || W > 32768 || H > 32768) return DCO_EINVAL;   // W*H < 2^31
    dco_dense_params p;
    if (pin) p = *pin;
    else dco_dense_params_default(&p);
    if (!(p.lambda_d >= 0.f) || !(p.lambda_s >= 0.f) || !(p.lambda_s2 >= 0.f) || !(p.tol > 0.f) ||
        p.max_iters < 0 || p.max_iters > 1000000)
        return DCO_EINVAL;
    DCO_CUDA(h, enter_device(h));
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    DCO_CUDA(h, cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone) {
        h->last_error = "dco_stereo_densify waits for its solve and cannot be captured";
        return DCO_EINVAL;
    }
    const size_t n = (size_t)W * H;
    // grid-stride kernels: at most 8 resident blocks per multiprocessor
    int nsm = 0;
    DCO_CUDA(h, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
    const int nblk = (int)std::min<size_t>((n + kDnBlock - 1) / kDnBlock, (size_t)std::max(nsm, 1) * 8);
    // workspace: r, z, p0, p1, Ap, wr, wd, diag, b; block partials; scalars
    const size_t fl = align_up(4 * n);
    const size_t off_part = 9 * fl, off_sc = off_part + align_up(16 * (size_t)nblk);
    dco_status st = ensure_ws(h, off_sc + align_up(sizeof(DnScalars)));
    if (st != DCO_OK) return st;
    if (!h->dn_pin) {
        DCO_CUDA(h, cudaMallocHost((void **)&h->dn_pin, 2 * sizeof(int)));
        for (auto &e : h->dn_ev) DCO_CUDA(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    DnArgs a;
    std::memset(&a, 0, sizeof a);   // padding included: the bytes key the captured graph
    a.ds = d_sparse; a.dpre = d_pre; a.mf = m_fuse; a.mi = m_int; a.contour = contour;
    float *f = ws_ptr<float>(h, 0);
    auto arr = [&](int k) { return reinterpret_cast<float *>(reinterpret_cast<char *>(f) + k * fl); };
    a.x = d_out; a.r = arr(0); a.z = arr(1); a.p[0] = arr(2); a.p[1] = arr(3); a.ap = arr(4);
    a.wr = arr(5); a.wd = arr(6); a.dg = arr(7); a.b = arr(8);
    a.part = ws_ptr<double>(h, off_part);
    a.sc = ws_ptr<DnScalars>(h, off_sc);
    a.W = W; a.H = H; a.nblk = nblk;
    a.lambda_d = p.lambda_d; a.lambda_s = p.lambda_s; a.lambda_s2 = p.lambda_s2;
    a.tol2 = (double)p.tol * p.tol;
    {
        ProfScope ps(h, s, "k_dn_setup");
        launch_pdl(k_dn_setup, dim3(nblk), dim3(kDnBlock), 0, s, a);
    }
    {
        ProfScope ps(h, s, "k_dn_init");
        launch_pdl(k_dn_init, dim3(nblk), dim3(kDnBlock), 0, s, a);
    }
    DCO_CUDA(h, cudaGetLastError());
    // Iterations run in batches of kDnIters, each closed by the residual
    // replacement, the true-residual test and a copy of the (sticky) done
    // flag to pinned memory.  A batch is one CUDA graph launch (captured once
    // per argument set on a private stream; per-kernel profiling uses plain
    // launches instead); the host keeps one batch queued ahead and stops
    // enqueuing once the flag of an earlier batch reads 1.
    constexpr int kDnIters = 16;   // even: buffer parity repeats per batch
    auto enqueue = [&](cudaStream_t q, int it0, int m, bool prof) -> cudaError_t {
        for (int k = 0; k < m; k++) {
            const int it = it0 + k;
            {
                ProfScope ps(h, q, prof ? "k_dn_ap" : nullptr);
                launch_pdl(k_dn_ap, dim3(nblk), dim3(kDnBlock), 0, q, a, it);
            }
            {
                ProfScope ps(h, q, prof ? "k_dn_upd" : nullptr);
                launch_pdl(k_dn_upd, dim3(nblk), dim3(kDnBlock), 0, q, a, it);
            }
        }
        {
            ProfScope ps(h, q, prof ? "k_dn_resid" : nullptr);
            launch_pdl(k_dn_resid, dim3(nblk), dim3(kDnBlock), 0, q, a);
        }
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->dn_pin, &a.sc->done, sizeof(int), cudaMemcpyDeviceToHost, q);
        return e;
    };
    const bool graph = !h->profiling;
    if (graph) {
        const unsigned char *ka = reinterpret_cast<const unsigned char *>(&a);
        if (!h->dn_exec || h->dn_key.size() != sizeof a || std::memcmp(h->dn_key.data(), ka, sizeof a)) {
            if (h->dn_exec) {
                cudaGraphExecDestroy(h->dn_exec);
                h->dn_exec = nullptr;
            }
            if (!h->dn_stream) DCO_CUDA(h, cudaStreamCreateWithFlags(&h->dn_stream, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            DCO_CUDA(h, cudaStreamBeginCapture(h->dn_stream, cudaStreamCaptureModeThreadLocal));
            const cudaError_t e = enqueue(h->dn_stream, 0, kDnIters, false);
            const cudaError_t e2 = cudaStreamEndCapture(h->dn_stream, &g);
            DCO_CUDA(h, e);
            DCO_CUDA(h, e2);
            const cudaError_t e3 = cudaGraphInstantiate(&h->dn_exec, g, 0);
            cudaGraphDestroy(g);
            DCO_CUDA(h, e3);
            h->dn_key.assign(ka, ka + sizeof a);
        }
    }
    *h->dn_pin = 0;
    int it = 0, nb = 0;
    bool stop = false;
    while (it < p.max_iters && !stop) {
        const int m = std::min(kDnIters, p.max_iters - it);
        if (graph && m == kDnIters) {
            DCO_CUDA(h, cudaGraphLaunch(h->dn_exec, s));
            h->launches += 2 * kDnIters + 1;
        } else {
            DCO_CUDA(h, enqueue(s, it, m, true));
        }
        it += m;
        DCO_CUDA(h, cudaEventRecord(h->dn_ev[nb & 1], s));
        if (nb > 0) {
            DCO_CUDA(h, cudaEventSynchronize(h->dn_ev[(nb - 1) & 1]));
            stop = *reinterpret_cast<volatile int *>(h->dn_pin) != 0;
        }
        nb++;
    }
    DnScalars sc{};
    DCO_CUDA(h, cudaMemcpyAsync(&sc, a.sc, sizeof sc, cudaMemcpyDeviceToHost, s));
    DCO_CUDA(h, cudaStreamSynchronize(s));
    h->dn_iters = sc.iters;
    h->dn_relres = sc.bb > 0.0 ? std::sqrt(sc.rr / sc.bb) : 0.0;
    return DCO_OK;
}

dco_status dco_stereo_densify_stats(dco_stereo *h, int *iters, double *rel_residual)
{
    if (!h) return DCO_EINVAL;
    if (iters) *iters = h->dn_iters;
    if (rel_residual) *rel_residual = h->dn_relres;
    return DCO_OK;
}

}  // extern "C"
