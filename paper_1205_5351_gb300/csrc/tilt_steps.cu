// Step kernels: one step of the solver on given inputs, with the solver's own device code
// (the step entry points of the C ABI use them for per-step parity), and their launchers.
#include "tilt_cayley.cuh"
#include "tilt_launch.h"
#include "tilt_solver.cuh"

namespace tilt {

__global__ void __launch_bounds__(NT, 1) warp_step_kernel(WarpArgs a) {
    extern __shared__ __align__(256) unsigned char smem_raw[];
    SmemLayout L = carve_smem(smem_raw);
    const Dims d = make_dims(a.m, a.n, a.ttype);
    k1_warp_jacobian(a.img, a.ld, a.H, a.W, d, a.ttype, a.tau, a.Dhat, a.J, L.sc);
    if (threadIdx.x == 0) {
        a.out->norm = L.sc->scal[0];
        a.out->oob = L.sc->iscal[0];
    }
}

__global__ void __launch_bounds__(NT, 1) gram_step_kernel(GramArgs a) {
    extern __shared__ __align__(256) unsigned char smem_raw[];
    SmemLayout L = carve_smem(smem_raw);
    const Dims d = make_dims(a.m, a.n, a.ttype);
    const bool ok = k5_gram(d, a.ttype, a.tau, a.Dhat, a.J, L.sc);
    if (threadIdx.x == 0) {
        a.out->status = ok ? 0 : -2;
        for (int k = 0; k < 3 * PMAX; ++k) a.out->Q[k] = L.sc->Q[k];
        for (int k = 0; k < PMAX * PMAX; ++k) {
            a.out->G[k] = L.sc->G[k];
            a.out->Gi[k] = L.sc->Gi[k];
        }
    }
}

__global__ void __launch_bounds__(NT, 1) svt_step_kernel(SvtArgs a) {
    extern __shared__ __align__(256) unsigned char smem_raw[];
    SmemLayout L = carve_smem(smem_raw);
    tc_setup(&L.sc->tc, TC_TMEM_COLS);
    const Dims d = make_dims(a.m, a.n, 0);
    float *B, *V;
    unsigned char* stage;
    if (a.smem_svd) {
        B = L.svd;
        V = B + (size_t)d.ldb * d.Cp;
        stage = reinterpret_cast<unsigned char*>(V + (size_t)d.ldv * d.Cp);
    } else {
        B = a.Bg;
        V = a.Vg;
        stage = reinterpret_cast<unsigned char*>(L.svd);
    }
    int reorth = 0;
    if (!a.Vio) {
        for (int e = threadIdx.x; e < d.ldb * d.Cp; e += NT) {
            const int r = e % d.ldb, c = e / d.ldb;
            B[e] = (r < d.R && c < d.C) ? a.M[(size_t)c * d.R + r] : 0.f;
        }
        __syncthreads();
        set_identity(V, d.ldv, d.Cp);
    } else {
        // warm start from the caller's V (padding: identity), re-orthonormalised in FP64 when it
        // has drifted, then B = M V with the solver's product
        for (int e = threadIdx.x; e < d.ldv * d.Cp; e += NT) {
            const int r = e % d.ldv, c = e / d.ldv;
            V[e] = (r < d.C && c < d.C) ? a.Vio[(size_t)c * d.C + r] : (r == c ? 1.f : 0.f);
        }
        __syncthreads();
        if (v_drift(V, d.ldv, d.C, L.sc) > 1e-4f) {
            v_reorth_fp64(V, d.ldv, d.C, L.sc);
            reorth = 1;
        }
        for (int e = threadIdx.x; e < d.ldb * d.Cp; e += NT) B[e] = 0.f;
        __syncthreads();
        const float* Mx = a.M;
        const int R = d.R, ldv = d.ldv, ldb = d.ldb;
        auto la = [=](int r, int j) { return Mx[(size_t)j * R + r]; };
        auto lb = [=](int j, int c) { return V[(size_t)c * ldv + j]; };
        auto ep = [=](int r, int c, float v) { B[(size_t)c * ldb + r] = v; };
        if (use_tc_products(d)) {
            if (!tc_gemm<NT, false, true>(d.R, d.C, d.C, la, lb, ep, stage, TC_KC, 1, &L.sc->tc)) {
                if (threadIdx.x == 0) a.out->status = -5;
                tc_teardown(&L.sc->tc, TC_TMEM_COLS);
                return;
            }
        } else {
            for (int e = threadIdx.x; e < d.R * d.C; e += NT) {
                const int r = e % d.R, c = e / d.R;
                float acc = 0.f;
                for (int j = 0; j < d.C; ++j) acc = fmaf(la(r, j), lb(j, c), acc);
                ep(r, c, acc);
            }
            __syncthreads();
        }
    }
    int sw;
    if (jsched_order(a.jsched) == 2) {
        sw = k2_jacobi_staged<4>(B, d.ldb, V, d.ldv, d.R, d.C, jacobi_tol(d.R), 60, L.sc->flag, jsched_width(a.jsched),
                                 reinterpret_cast<float*>(stage), &L.sc->tc, L.w);
    } else {
        sw = k2_jacobi<4>(B, d.ldb, V, d.ldv, d.R, d.C, jacobi_tol(d.R), 60, L.sc->flag, jsched_width(a.jsched),
                          jsched_order(a.jsched), L.w);
    }
    if (sw < 0) {
        if (threadIdx.x == 0) a.out->status = -5;
        tc_teardown(&L.sc->tc, TC_TMEM_COLS);
        return;
    }
    svt_weights(B, d.ldb, d.R, d.C, a.eps, L.sigma, L.w, L.kept, L.sc);
    const int nk = L.sc->iscal[1];
    // the solver's SVT: coefficients Z = diag(w / sigma^2) B_K^T M and A = B_K Z, on the tensor
    // cores for the windows where the solver uses them
    const bool tc = use_tc_products(d);
    bool ok = true;
    if (tc)
        ok = svt_coeffs_tc(a.M, d.R, B, d.ldb, d.R, d.C, L.sigma, L.w, L.kept, nk, a.Zg, d.Cp, stage, 1, &L.sc->tc);
    else
        svt_left_coeffs(a.M, d.R, B, d.ldb, d.R, d.C, L.sigma, L.w, L.kept, nk, a.Zg, d.Cp);
    float* A = a.A;
    const int R = d.R;
    auto put = [=](int r, int c, float v) { A[(size_t)c * R + r] = v; };
    if (nk > 0 && tc && ok) {
        const float* Zg = a.Zg;
        const int* kept = L.kept;
        const int ldb = d.ldb, ldz = d.Cp;
        auto la = [=](int r, int q) { return B[(size_t)kept[q] * ldb + r]; };
        auto lb = [=](int q, int c) { return Zg[(size_t)q * ldz + c]; };
        ok = tc_gemm<NT, false, false>(d.R, d.C, nk, la, lb, put, stage, TC_KC, 1, &L.sc->tc);
    } else if (!tc) {
        for (int e = threadIdx.x; e < d.S; e += NT) {
            const int r = e % d.R, c = e / d.R;
            float acc = 0.f;
            for (int q = 0; q < nk; ++q) acc = fmaf(B[(size_t)L.kept[q] * d.ldb + r], a.Zg[(size_t)q * d.Cp + c], acc);
            A[e] = acc;
        }
    } else if (nk == 0) {
        for (int e = threadIdx.x; e < d.S; e += NT) A[e] = 0.f;
    }
    for (int k = threadIdx.x; k < d.C; k += NT) a.sigma[k] = L.sigma[k];
    if (a.Vio)
        for (int e = threadIdx.x; e < d.C * d.C; e += NT) a.Vio[e] = V[(size_t)(e / d.C) * d.ldv + e % d.C];
    if (threadIdx.x == 0) {
        a.out->sweeps = sw;
        a.out->reorth = reorth;
        a.out->status = ok ? 0 : -5;
    }
    tc_teardown(&L.sc->tc, TC_TMEM_COLS);
}

__global__ void __launch_bounds__(NT, 1) inner_step_kernel(InnerArgs a) {
    extern __shared__ __align__(256) unsigned char smem_raw[];
    SmemLayout L = carve_smem(smem_raw);
    tc_setup(&L.sc->tc, TC_TMEM_COLS);
    const Dims d = make_dims(a.m, a.n, a.ttype);
    SvdBufs buf;
    if (a.smem_svd) {
        buf.B = L.svd;
        buf.V = buf.B + (size_t)d.ldb * d.Cp;
        buf.T = buf.V + (size_t)d.ldv * d.Cp;
        buf.stage = reinterpret_cast<unsigned char*>(buf.T + (size_t)d.ldb * d.Cp);
    } else {
        buf.B = a.Bg;
        buf.V = a.Vg;
        buf.T = a.Tg;
        buf.stage = reinterpret_cast<unsigned char*>(L.svd);
    }
    buf.Z = a.Zg;
    buf.nbuf = 1;
    buf.tc = use_tc_products(d);
    {
        const size_t nb = (size_t)d.ldb * d.Cp, nv = (size_t)d.ldv * d.Cp;
        for (size_t e = threadIdx.x; e < nb; e += NT) { buf.B[e] = 0.f; buf.T[e] = 0.f; }
        for (size_t e = threadIdx.x; e < nv; e += NT) buf.V[e] = 0.f;
        for (int e = threadIdx.x; e < d.S; e += NT) a.Mp[e] = 0.f;
    }
    __syncthreads();
    if (!k5_gram(d, a.ttype, a.tau, a.Dhat, a.J, L.sc, a.use_q != 0)) {
        if (threadIdx.x == 0) a.out->status = -2;
        tc_teardown(&L.sc->tc, TC_TMEM_COLS);
        return;
    }
    double mu0 = a.mu0;
    if (!(mu0 > 0.0)) mu0 = 1.25 / spectral_norm(a.Dhat, d, L.sigma, L.w, L.sc);
    const double lam = a.prm.lam > 0.0 ? a.prm.lam : 1.0 / sqrt((double)max(a.m, a.n));
    bool haveV = false;
    __shared__ Result cyc;
    if (threadIdx.x == 0) cyc.cyc_elem = cyc.cyc_svd = cyc.cyc_recon = cyc.cyc_warp = cyc.cyc_other = 0;
    __syncthreads();
    InnerOut io = k_inner<4>(d, a.prm, lam, mu0, a.Dhat, a.J, a.A, a.E, a.Y, a.Mp, buf, haveV, L, &cyc,
                             a.jsched, nullptr, a.Cay);
    if (threadIdx.x == 0) {
        a.out->status = io.tc_timeout ? -5 : io.bad ? -1 : 0;
        a.out->iters = io.iters;
        a.out->sweeps = io.sweeps;
        a.out->c1 = io.c1;
        a.out->c2 = io.c2;
        a.out->mu = io.mu_last;
        a.out->accepted = io.cayley;
        for (int k = 0; k < PMAX; ++k) a.out->dtau[k] = k < a.ttype ? L.sc->cvec[k] : 0.0;
    }
    tc_teardown(&L.sc->tc, TC_TMEM_COLS);
}

// The ADM of Zhang et al. (the comparison method of Sec. 2.2) on one problem: D, J given.
__global__ void __launch_bounds__(NT, 1) adm_step_kernel(AdmArgs a) {
    extern __shared__ __align__(256) unsigned char smem_raw[];
    SmemLayout L = carve_smem(smem_raw);
    tc_setup(&L.sc->tc, TC_TMEM_COLS);
    const Dims d = make_dims(a.m, a.n, a.p);
    SvdBufs buf;
    if (a.smem_svd) {
        buf.B = L.svd;
        buf.V = buf.B + (size_t)d.ldb * d.Cp;
        buf.T = buf.V + (size_t)d.ldv * d.Cp;
        buf.stage = reinterpret_cast<unsigned char*>(buf.T + (size_t)d.ldb * d.Cp);
    } else {
        buf.B = a.Bg;
        buf.V = a.Vg;
        buf.T = a.Tg;
        buf.stage = reinterpret_cast<unsigned char*>(L.svd);
    }
    buf.Z = a.Zg;
    buf.nbuf = 1;
    buf.tc = use_tc_products(d);
    {
        const size_t nb = (size_t)d.ldb * d.Cp, nv = (size_t)d.ldv * d.Cp;
        for (size_t e = threadIdx.x; e < nb; e += NT) { buf.B[e] = 0.f; buf.T[e] = 0.f; }
        for (size_t e = threadIdx.x; e < nv; e += NT) buf.V[e] = 0.f;
    }
    __syncthreads();
    if (!k5_gram(d, 0, nullptr, a.D, a.J, L.sc, false)) {
        if (threadIdx.x == 0) a.out->status = -2;
        tc_teardown(&L.sc->tc, TC_TMEM_COLS);
        return;
    }
    double mu0 = a.mu0;
    if (!(mu0 > 0.0)) mu0 = 1.25 / spectral_norm(a.D, d, L.sigma, L.w, L.sc);
    const AdmOut o = k_inner_adm<4, true>(d, a.lam, a.tol, a.rho, mu0, a.max_iter, a.D, a.J, a.A, a.E, a.Y, buf, L,
                                          a.jsched);
    if (threadIdx.x == 0) {
        a.out->status = o.tc_timeout ? -5 : o.bad ? -1 : (o.converged ? 0 : 2);
        a.out->iters = o.iters;
        a.out->sweeps = o.sweeps;
        a.out->c1 = o.residual;
        a.out->mu = o.mu_last;
        for (int k = 0; k < PMAX; ++k) a.out->dtau[k] = k < a.p ? L.sc->dtau[k] : 0.0;
    }
    tc_teardown(&L.sc->tc, TC_TMEM_COLS);
}

// One step of Algorithm 2 (the SVD warm start of Sec. 5) on given factors.  Workspace:
// the Cayley buffers, then M and V at the strides the step uses (ldb, ldv).
__global__ void __launch_bounds__(NT, 1) cayley_step_kernel(CayArgs a) {
    extern __shared__ __align__(256) unsigned char smem_raw[];
    SmemLayout L = carve_smem(smem_raw);
    const Dims d = make_dims(a.m, a.n, 0);
    const int R = d.R, C = d.C;
    CayBufs cb = carve_cayley(a.work, d);
    float* Mx = a.work + cayley_floats(d);
    float* Vw = Mx + (size_t)d.ldb * d.Cp;
    for (int e = threadIdx.x; e < d.ldb * C; e += NT) {
        const int r = e % d.ldb, c = e / d.ldb;
        Mx[e] = r < R ? a.M[(size_t)c * R + r] : 0.f;
        cb.U[e] = r < R ? a.U[(size_t)c * R + r] : 0.f;
    }
    for (int e = threadIdx.x; e < d.ldv * C; e += NT) {
        const int r = e % d.ldv, c = e / d.ldv;
        Vw[e] = r < C ? a.V[(size_t)c * C + r] : 0.f;
    }
    for (int i = threadIdx.x; i < C; i += NT) cb.S[i] = a.S[i];
    __syncthreads();
    const CayleyOut o = cayley_step(d, Mx, cb, Vw, L.sc);
    if (o.accepted) {
        for (int e = threadIdx.x; e < R * C; e += NT) a.U[e] = cb.U[(size_t)(e / R) * d.ldb + e % R];
        for (int e = threadIdx.x; e < C * C; e += NT) a.V[e] = Vw[(size_t)(e / C) * d.ldv + e % C];
        for (int i = threadIdx.x; i < C; i += NT) a.S[i] = cb.S[i];
    }
    if (threadIdx.x == 0) {
        a.out->accepted = o.accepted ? 1 : 0;
        a.out->cay[0] = o.f1;
        a.out->cay[1] = o.f2;
        a.out->cay[2] = o.t;
        a.out->cay[3] = o.f0;
        a.out->cay[4] = o.ft;
        a.out->status = 0;
    }
}

cudaError_t configure_step_kernels(size_t max_smem) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(svt_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem)))
        return e;
    if ((e = cudaFuncSetAttribute(inner_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem)))
        return e;
    return cudaFuncSetAttribute(adm_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem);
}

cudaError_t launch_warp_step(const WarpArgs& a, cudaStream_t st) {
    warp_step_kernel<<<1, NT, smem_head_bytes(), st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gram_step(const GramArgs& a, cudaStream_t st) {
    gram_step_kernel<<<1, NT, smem_head_bytes(), st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_svt_step(const SvtArgs& a, size_t smem, cudaStream_t st) {
    svt_step_kernel<<<1, NT, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_inner_step(const InnerArgs& a, size_t smem, cudaStream_t st) {
    inner_step_kernel<<<1, NT, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cayley_step(const CayArgs& a, cudaStream_t st) {
    cayley_step_kernel<<<1, NT, smem_head_bytes(), st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adm_step(const AdmArgs& a, size_t smem, cudaStream_t st) {
    adm_step_kernel<<<1, NT, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace tilt
