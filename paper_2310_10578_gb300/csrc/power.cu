// power.cu -- received power in dBm from the evaluated field.
//
// The paper reports received-power maps and line cuts in dBm for a 40 dBm
// omnidirectional transmitter (Sec. IV).  The field out of rt_evaluate is
// normalised so that free space gives |E| = 1/R (1 V at 1 m); for an
// isotropic receiving antenna the Friis form then gives
//     P_r[dBm] = P_t[dBm] + 20 log10(lambda / (4 pi)) + 20 log10 |E . p|,
// with p the receiving antenna's unit polarisation (|E| itself when no
// polarisation is given: the power summed over polarisations).  No field
// (a receiver with no path, or inside a body) gives -inf.
#include "internal.h"

namespace creep {

namespace {

__global__ void k_power_dbm(const float *__restrict__ e, int n_f, int n_rx, const float *__restrict__ c0,
                            float px, float py, float pz, int use_pol, float *__restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n_f * n_rx) return;
    const int f = (int)(i / n_rx), r = (int)(i - (long long)f * n_rx);
    float m2;
    const float2 *E = reinterpret_cast<const float2 *>(e);
    const float2 ex = E[((size_t)f * 3 + 0) * n_rx + r], ey = E[((size_t)f * 3 + 1) * n_rx + r],
                 ez = E[((size_t)f * 3 + 2) * n_rx + r];
    if (use_pol) {
        const float re = ex.x * px + ey.x * py + ez.x * pz, im = ex.y * px + ey.y * py + ez.y * pz;
        m2 = re * re + im * im;
    } else {
        m2 = ex.x * ex.x + ex.y * ex.y + ey.x * ey.x + ey.y * ey.y + ez.x * ez.x + ez.y * ez.y;
    }
    // 10 log10 |E|^2 + (P_t + 20 log10(lambda / 4 pi)) of this frequency
    out[i] = (m2 > 0.0f) ? 10.0f * log10f(m2) + c0[f] : -INFINITY;
}

}  // namespace

int launch_power_dbm(const float *e_out, int n_f, int n_rx, const float *c0_dev, const float pol[3], float *p_out,
                     cudaStream_t st) {
    const long long n = (long long)n_f * n_rx;
    if (n == 0) return RT_OK;
    float p[3] = {0.f, 0.f, 0.f};
    if (pol) {
        const double nn = sqrt((double)pol[0] * pol[0] + (double)pol[1] * pol[1] + (double)pol[2] * pol[2]);
        for (int k = 0; k < 3; ++k) p[k] = (float)(pol[k] / nn);
    }
    k_power_dbm<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(e_out, n_f, n_rx, c0_dev, p[0], p[1], p[2], pol ? 1 : 0,
                                                          p_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("k_power_dbm: ") + cudaGetErrorString(e));
        return RT_ERR_CUDA;
    }
    return RT_OK;
}

}  // namespace creep
