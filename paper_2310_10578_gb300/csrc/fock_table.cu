// fock_table.cu -- device construction (FP64) of the Fock--Pekeris table and
// the residue-series constants used by the field kernel.
//
// Table: G_{s,h}(xi) = phat_{s,h}(xi) e^{-j xi^3/12} and dG/dxi at
// xi_j = XI_LO + j * XI_STEP, j = 0 .. FOCK_N - 1, covering [XI_LO, XI_HI];
// and P_{s,h}(xi) = phat - c/xi with dP/dxi on [XI_HI, XI_P] (the FP32
// fields' second segment; from XI_PRES on by the residue series).
// The e^{-j xi^3/12} factor removes the geometrical-optics phase of the lit
// side (phat ~ sqrt(-xi/4) e^{j xi^3/12} as xi -> -inf), leaving a slowly
// varying function for cubic Hermite interpolation.
//
// Quadrature (see fock_math.cuh): tau in [0, 9] on the real axis; the
// negative branch in x = -tau deformed by angle pi/4 into the upper half
// plane: for xi >= 0 straight from 0; for xi in [-n, -n+1) along the real
// axis to x1 = n^2/4 + 3/2 (past the stationary point xi^2/4) and then along
// x1 + u e^{j pi/4}.  Composite 20-point Gauss-Legendre, panels <= 0.6.
//
// Residue constants: the first 8 zeros -alpha_n of Ai and -beta_n of Ai'
// (asymptotic first guesses, A&S 10.4.94-95, polished by Newton with the
// device Airy functions) and the residues 1/Ai'(-alpha_n)^2,
// 1/(beta_n Ai(-beta_n)^2).
#include <cuda_runtime.h>
#include <mutex>
#include <string>
#include <vector>

#include "fock_math.cuh"
#include "internal.h"

namespace creep {

static const int GL_N = 20;
static const double PANEL = 0.6;
static const double TAU_POS_MAX = 9.0;
static const double RAY_LEN_POS = 9.0;
static const double RAY_LEN_NEG = 16.0;

// Gauss-Legendre nodes/weights on [-1, 1] by Newton on P_n.
static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            double dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1; p1 = p2;
        }
        double dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Append composite GL nodes along the straight path x = x0 + s e, s in [0, len];
// node in tau = -x, weight includes dx = e ds.
static void add_path(std::vector<cd> &tau, std::vector<cd> &wt, cd x0, cd e, double len, bool neg,
                     const std::vector<double> &gx, const std::vector<double> &gw) {
    int np = (int)ceil(len / PANEL);
    if (np < 1) np = 1;
    double h = len / np;
    for (int p = 0; p < np; ++p) {
        for (int i = 0; i < GL_N; ++i) {
            double s = (p + 0.5) * h + 0.5 * h * gx[i];
            cd x = x0 + e * s;
            tau.push_back(neg ? -x : x);
            wt.push_back(e * (0.5 * h * gw[i]));
        }
    }
}

__global__ void k_fock_integrands(const cd *tau, const cd *wt, int n_pos, int n, cd *Ws, cd *Wh) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    cd gs, gh;
    fock_integrands(tau[i], i < n_pos, &gs, &gh);
    Ws[i] = wt[i] * gs;
    Wh[i] = wt[i] * gh;
}

// One block per table node xi = xi0 + j XI_STEP: phat, dphat/dxi by summing
// the bucket's nodes; stored as G = phat e^{-j xi^3/12} and G' (p_form false)
// or as P = phat - c/xi and P' = phat' + c/xi^2 (p_form true, xi > 0).  In
// P form from XI_PRES on, P and P' come from the residue series instead:
// P = -e^{-j pi/12}/(2 sqrt(pi)) sum_n coef_n e^{-xi z_n}, z_n = a_n e^{j pi/6}
// (a_n the zeros alpha_n, beta_n; res as k_airy_zeros writes it).
__global__ void k_fock_table(const cd *tau, const cd *Ws, const cd *Wh, int n_pos, const int *neg_off,
                             int n_tab, double xi0, bool p_form, const double *res,
                             double *out /* [n_tab][2 kinds][4] = G.re, G.im, G'.re, G'.im (or P, P') */) {
    int j = blockIdx.x;
    if (j >= n_tab) return;
    double xi = xi0 + j * XI_STEP;
    if (p_form && xi >= XI_PRES) {
        if (threadIdx.x == 0) {
            const cd pre = -cpolar(0.5 / sqrt(M_PI), -M_PI / 12.0);
            for (int k = 0; k < 2; ++k) {
                cd s = C(0), ds = C(0);
                for (int n = 0; n < FOCK_NRES; ++n) {
                    const double a = res[(2 * k) * FOCK_NRES + n], coef = res[(2 * k + 1) * FOCK_NRES + n];
                    const cd z = C(a * (0.5 * sqrt(3.0)), a * 0.5);
                    const cd t = cexp_(-(z * xi)) * coef;
                    s = s + t;
                    ds = ds - z * t;
                }
                const cd P = pre * s, dP = pre * ds;
                out[(j * 2 + k) * 4 + 0] = P.x;
                out[(j * 2 + k) * 4 + 1] = P.y;
                out[(j * 2 + k) * 4 + 2] = dP.x;
                out[(j * 2 + k) * 4 + 3] = dP.y;
            }
        }
        return;
    }
    int b = (xi >= 0.0) ? 0 : (int)ceil(-xi);
    int lo = neg_off[b], hi = neg_off[b + 1];
    int cnt = n_pos + (hi - lo);
    cd s0 = C(0), s1 = C(0), d0 = C(0), d1 = C(0);
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        int i = (t < n_pos) ? t : lo + (t - n_pos);
        cd e = cexp_(C(0.0, -1.0) * xi * tau[i]);        // e^{-j xi tau}
        cd mjt = C(0.0, -1.0) * tau[i];                  // -j tau
        s0 = s0 + Ws[i] * e;
        s1 = s1 + Wh[i] * e;
        d0 = d0 + Ws[i] * mjt * e;
        d1 = d1 + Wh[i] * mjt * e;
    }
    __shared__ double red[8][256];
    red[0][threadIdx.x] = s0.x; red[1][threadIdx.x] = s0.y;
    red[2][threadIdx.x] = s1.x; red[3][threadIdx.x] = s1.y;
    red[4][threadIdx.x] = d0.x; red[5][threadIdx.x] = d0.y;
    red[6][threadIdx.x] = d1.x; red[7][threadIdx.x] = d1.y;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 8; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        cd pre = cpolar(1.0 / sqrt(M_PI), -M_PI / 4.0);
        cd ph[2] = {pre * C(red[0][0], red[1][0]), pre * C(red[2][0], red[3][0])};
        cd dph[2] = {pre * C(red[4][0], red[5][0]), pre * C(red[6][0], red[7][0])};
        if (p_form) {
            const cd c = cpolar(0.5 / sqrt(M_PI), -M_PI / 4.0);   // e^{-j pi/4} / (2 sqrt(pi))
            for (int k = 0; k < 2; ++k) {
                cd P = ph[k] - c * (1.0 / xi), dP = dph[k] + c * (1.0 / (xi * xi));
                out[(j * 2 + k) * 4 + 0] = P.x;
                out[(j * 2 + k) * 4 + 1] = P.y;
                out[(j * 2 + k) * 4 + 2] = dP.x;
                out[(j * 2 + k) * 4 + 3] = dP.y;
            }
            return;
        }
        cd rot = cpolar(1.0, -xi * xi * xi / 12.0);          // e^{-j xi^3/12}
        for (int k = 0; k < 2; ++k) {
            cd G = ph[k] * rot;
            cd dG = (dph[k] - C(0.0, xi * xi / 4.0) * ph[k]) * rot;
            out[(j * 2 + k) * 4 + 0] = G.x;
            out[(j * 2 + k) * 4 + 1] = G.y;
            out[(j * 2 + k) * 4 + 2] = dG.x;
            out[(j * 2 + k) * 4 + 3] = dG.y;
        }
    }
}

// Ai(-x), Ai'(-x) for x > 0.  For x >= 7.5 through Ai(z) = -w Ai(w z) - w^2 Ai(w^2 z)
// (DLMF 9.2.12) at arguments of modulus x and argument -+pi/3.
__host__ __device__ inline void airy_negreal(double x, double *ai, double *aip) {
    if (x < 7.5) {
        airy_t a = airy(C(-x, 0.0));
        *ai = a.ai.x;
        *aip = a.aip.x;
        return;
    }
    cd w = cpolar(1.0, 2.0 * M_PI / 3.0), wb = cpolar(1.0, -2.0 * M_PI / 3.0);
    airy_t a1 = airy(cpolar(x, -M_PI / 3.0)), a2 = airy(cpolar(x, M_PI / 3.0));
    cd s1 = cexp_(-a1.zeta), s2 = cexp_(-a2.zeta);
    cd v = -(w * a1.ai * s1) - (wb * a2.ai * s2);
    cd d = -(wb * a1.aip * s1) - (w * a2.aip * s2);
    *ai = v.x;
    *aip = d.x;
}

__global__ void k_airy_zeros(double *res /* [4][8] */) {
    int n = threadIdx.x;
    if (n >= 2 * FOCK_NRES) return;
    int s = (n % FOCK_NRES) + 1;
    bool hard = n >= FOCK_NRES;
    double t = hard ? 3.0 * M_PI * (4.0 * s - 3.0) / 8.0 : 3.0 * M_PI * (4.0 * s - 1.0) / 8.0;
    double t2 = 1.0 / (t * t);
    double x = pow(t, 2.0 / 3.0) * (hard ? (1.0 - 7.0 / 48.0 * t2 + 35.0 / 288.0 * t2 * t2)
                                         : (1.0 + 5.0 / 48.0 * t2 - 5.0 / 36.0 * t2 * t2));
    double ai, aip;
    for (int it = 0; it < 60; ++it) {
        airy_negreal(x, &ai, &aip);
        double dx = hard ? aip / (x * ai)   // d/dx Ai'(-x) = x Ai(-x)
                         : -ai / aip;       // d/dx Ai(-x) = -Ai'(-x)
        x -= dx;
        if (fabs(dx) < 1e-15 * x) break;
    }
    airy_negreal(x, &ai, &aip);
    if (!hard) {
        res[0 * FOCK_NRES + s - 1] = x;
        res[1 * FOCK_NRES + s - 1] = 1.0 / (aip * aip);
    } else {
        res[2 * FOCK_NRES + s - 1] = x;
        res[3 * FOCK_NRES + s - 1] = 1.0 / (x * ai * ai);
    }
}

#define CK(call)                                                                  \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            set_error(std::string("fock table: ") + #call + ": " + cudaGetErrorString(e_)); \
            goto fail;                                                            \
        }                                                                         \
    } while (0)

// Build the table on the current device; fills host copies in T.
int build_fock_table(FockHost *T) {
    std::vector<double> gx, gw;
    gauss_legendre(GL_N, gx, gw);
    std::vector<cd> tau, wt;
    add_path(tau, wt, C(0.0), C(1.0), TAU_POS_MAX, false, gx, gw);
    int n_pos = (int)tau.size();
    std::vector<int> off(FOCK_NBUCKET + 1);
    cd e4 = cpolar(1.0, M_PI / 4.0);
    for (int b = 0; b < FOCK_NBUCKET; ++b) {
        off[b] = (int)tau.size();
        if (b == 0) {
            add_path(tau, wt, C(0.0), e4, RAY_LEN_POS, true, gx, gw);
        } else {
            double x1 = b * b / 4.0 + 1.5;
            add_path(tau, wt, C(0.0), C(1.0), x1, true, gx, gw);
            add_path(tau, wt, C(x1), e4, RAY_LEN_NEG, true, gx, gw);
        }
    }
    off[FOCK_NBUCKET] = (int)tau.size();
    int n = (int)tau.size();
    cd *d_tau = nullptr, *d_wt = nullptr, *d_ws = nullptr, *d_wh = nullptr;
    int *d_off = nullptr;
    double *d_out = nullptr, *d_outp = nullptr, *d_res = nullptr;
    int rc = RT_ERR_CUDA;
    CK(cudaMalloc(&d_tau, sizeof(cd) * n));
    CK(cudaMalloc(&d_wt, sizeof(cd) * n));
    CK(cudaMalloc(&d_ws, sizeof(cd) * n));
    CK(cudaMalloc(&d_wh, sizeof(cd) * n));
    CK(cudaMalloc(&d_off, sizeof(int) * (FOCK_NBUCKET + 1)));
    CK(cudaMalloc(&d_out, sizeof(double) * FOCK_N * 8));
    CK(cudaMalloc(&d_outp, sizeof(double) * FOCK_NP * 8));
    CK(cudaMalloc(&d_res, sizeof(double) * 4 * FOCK_NRES));
    CK(cudaMemcpy(d_tau, tau.data(), sizeof(cd) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_wt, wt.data(), sizeof(cd) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_off, off.data(), sizeof(int) * (FOCK_NBUCKET + 1), cudaMemcpyHostToDevice));
    k_fock_integrands<<<(n + 127) / 128, 128>>>(d_tau, d_wt, n_pos, n, d_ws, d_wh);
    CK(cudaGetLastError());
    k_airy_zeros<<<1, 32>>>(d_res);
    CK(cudaGetLastError());
    k_fock_table<<<FOCK_N, 256>>>(d_tau, d_ws, d_wh, n_pos, d_off, FOCK_N, XI_LO, false, d_res, d_out);
    CK(cudaGetLastError());
    k_fock_table<<<FOCK_NP, 256>>>(d_tau, d_ws, d_wh, n_pos, d_off, FOCK_NP, XI_HI, true, d_res, d_outp);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    T->tab.resize(FOCK_N * 8);
    T->tabp.resize(FOCK_NP * 8);
    T->res.resize(4 * FOCK_NRES);
    CK(cudaMemcpy(T->tab.data(), d_out, sizeof(double) * FOCK_N * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(T->tabp.data(), d_outp, sizeof(double) * FOCK_NP * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(T->res.data(), d_res, sizeof(double) * 4 * FOCK_NRES, cudaMemcpyDeviceToHost));
    T->n_nodes = n;
    rc = RT_OK;
fail:
    cudaFree(d_tau); cudaFree(d_wt); cudaFree(d_ws); cudaFree(d_wh);
    cudaFree(d_off); cudaFree(d_out); cudaFree(d_outp); cudaFree(d_res);
    return rc;
}

}  // namespace creep
