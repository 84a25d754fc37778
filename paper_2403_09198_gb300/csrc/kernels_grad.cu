// kernels_grad.cu -- adjoint outer products for x = J^-1 b.
//
// With lambda = J^-T g the derivative of the solve with respect to the stored
// Jacobian is dL/dJ = -lambda x^T, restricted to what is stored:
//   gS[block (i,j)][entry (p,q)] = -lambda_i[p] x_j[q]          (pattern of S_ij)
//   gU[pair of (i,j)]            = -(v . x_j) lambda_i          (column_data)
//   gV[pair of (i,j)]            = -(u . lambda_i) x_j          (row_data)
// The dots v . x_j are pass 1 of the forward matvec on x and u . lambda_i pass 1
// of the transposed matvec on lambda, so both come from the matvec kernels.
#include <cuda_runtime.h>

#include "sts_internal.h"

namespace sts {
namespace {

// One warp per block, lanes over pattern entries; output in the public S layout.
__global__ void k_grad_S(double *gS, const double *lam, const double *x, const long long *soff,
                         const int *blk_row, const int *blk_col, const int *erow, const int *didx,
                         const int *oidx, int nnzb, int nnz_d, int ncp) {
    const int lane = threadIdx.x & 31;
    const long long k = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (k >= nnzb) return;
    const int i = blk_row[k], j = blk_col[k];
    const bool diag = i == j;
    const int nnz = diag ? nnz_d : (int)(soff[k + 1] - soff[k]);
    const int *rows = erow + (diag ? 0 : nnz_d);
    const int *cols = diag ? didx : oidx;
    double *g = gS + soff[k];
    for (int e = lane; e < nnz; e += 32)
        g[e] = -lam[(size_t)rows[e] * ncp + i] * x[(size_t)cols[e] * ncp + j];
}

// One thread per (pair, component).
__global__ void k_grad_UV(double *gU, double *gV, const double *lam, const double *x,
                          const double *cN, const double *cT, const int *pair_cN, const int *pair_cT,
                          const int *pair_row, const int *pair_col, int n_pairs, int b, int ncp) {
    const long long total = (long long)n_pairs * b;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int pr = (int)(t / b), p = (int)(t % b);
        const int i = pair_row[pr], j = pair_col[pr];
        gU[t] = -cN[pair_cN[pr]] * lam[(size_t)p * ncp + i];
        gV[t] = -cT[pair_cT[pr]] * x[(size_t)p * ncp + j];
    }
}

}  // namespace

sts_status grad(sts_jac_s *h, const double *lam, const double *x, double *gS, double *gU, double *gV) {
    if (!h->g_c) {
        // internal copies of lambda and x plus the transposed pair dots
        STS_TRY(dalloc(h, &h->g_c, (size_t)h->n_tiles * h->mv[1].n_dtasks * kTile + 1));
    }
    double *li = h->vin, *xi = h->vout;
    STS_TRY(to_internal64(h, lam, li));
    STS_TRY(to_internal64(h, x, xi));
    STS_TRY(mv_dots64(h, 0, xi, h->c64));     // v . x_j   (forward pass 1 on x)
    STS_TRY(mv_dots64(h, 1, li, h->g_c));     // u . lambda_i (transposed pass 1 on lambda)
    k_grad_S<<<(unsigned)((h->nnzb + 3) / 4), 128, 0, h->stream>>>(
        gS, li, xi, h->d_soff, h->g_blk_row, h->g_blk_col, h->g_erow, h->mv[0].pat_idx,
        h->mv[0].pat_idx + h->nnz_d, h->nnzb, h->nnz_d, h->ncp);
    STS_LAUNCHED();
    if (h->n_pairs > 0) {
        const long long total = (long long)h->n_pairs * h->b;
        long long g = (total + 255) / 256;
        if (g > 152 * 64) g = 152 * 64;
        k_grad_UV<<<(unsigned)g, 256, 0, h->stream>>>(gU, gV, li, xi, h->c64, h->g_c, h->g_pair_cN,
                                                      h->g_pair_cT, h->g_pair_row, h->g_pair_col,
                                                      h->n_pairs, h->b, h->ncp);
        STS_LAUNCHED();
    }
    return STS_OK;
}

}  // namespace sts
