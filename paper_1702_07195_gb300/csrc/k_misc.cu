// Query-profile construction (paper Section 4.3, the Query Profile of Rognes & Seeberg):
// one int16 row per alphabet code d holding SM(q_i, d) for every query position i, biased by
// Goe (see QueryDesc), plus a row for the dummy padding code and padded rows scoring 0.
#include "swgb_device.cuh"

namespace swgb {

namespace {

__global__ void k_build_qp(const uint8_t* __restrict__ queries, const int64_t* __restrict__ qoff,
                           const int8_t* __restrict__ matrix, int32_t A, int32_t bias,
                           const int64_t* __restrict__ qp_off, const int32_t* __restrict__ mpad,
                           int16_t* __restrict__ qp, Control* ctrl) {
    const int q = blockIdx.z;
    const int d = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int m_pad = mpad[q];
    if (i >= m_pad) return;
    const int64_t q0 = qoff[q];
    const int m = static_cast<int>(qoff[q + 1] - q0);
    int s = 0;
    if (d < A && i < m) {
        const int code = queries[q0 + i];
        if (code < A)
            s = matrix[code * A + d];
        else if (d == 0)
            atomicOr(&ctrl->status, 1u);   // reported by the host after the search
    }
    qp[qp_off[q] + static_cast<int64_t>(d) * m_pad + i] = static_cast<int16_t>(s + bias);
}

}  // namespace

cudaError_t launch_build_qp(const uint8_t* d_queries, const int64_t* d_qoff, int32_t nq,
                            const int8_t* d_matrix, int32_t A, int32_t bias,
                            const int64_t* d_qp_off, const int32_t* d_mpad, int16_t* d_qp,
                            int64_t max_mpad, Control* ctrl, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    const int threads = 256;
    dim3 grid(static_cast<unsigned>((max_mpad + threads - 1) / threads),
              static_cast<unsigned>(A + 1), static_cast<unsigned>(nq));
    k_build_qp<<<grid, threads, 0, st>>>(d_queries, d_qoff, d_matrix, A, bias, d_qp_off, d_mpad,
                                         d_qp, ctrl);
    return cudaGetLastError();
}

}  // namespace swgb
