/*
 * oracle.c -- plain, slow FP64 CPU oracle for the block r1-sparse Jacobian path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
 * Python binding) links, loads or calls this file; only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark do.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * Every routine computes a plain definition, with no blocking or fusion:
 *
 *   Dense block assembly (Section 4.3 "Overall Structure", Section 5.1 BR1-BSR
 *   format): every stored block is  D_ij = S_ij + sum_k u_ijk v_ijk^T,  with
 *   S_ij scattered from its b x b CSR pattern and the rank-one pairs of block
 *   (i,j) taken from column_data (U) / row_data (V) in pair order.
 *
 *   Matvec (Section 3.4, standard block-sparse representation; Section 5.2):
 *   y_i = sum_j D_ij x_j, row by row; transposed: y_j = sum_i D_ij^T x_i.
 *
 *   Block-Jacobi (Section 6): M = blockdiag(A)^-1, each diagonal block D_ii
 *   factored by textbook LU with partial pivoting (Doolittle, unit lower L),
 *   z_i = D_ii^-1 x_i, or D_ii^-T x_i for the transposed operator.
 *
 *   Adjoint outer products (derivative of x = J^-1 b): with J^T lambda = g,
 *   dL/dS_ij[p][q] = -lambda_i[p] x_j[q] on the pattern,
 *   dL/du = -(v . x_j) lambda_i,  dL/dv = -(u . lambda_i) x_j.
 *
 * Data layout (all host arrays, row-major):
 *   block_indptr[nc+1], block_indices[nnzb]   block CSR of the mesh (incl. diagonal)
 *   d_indptr[b+1], d_indices[nnz_d]           pattern of every diagonal block
 *   o_indptr[b+1], o_indices[nnz_o]           pattern of every off-diagonal block
 *   pair_indptr[nnzb+1]                       pairs of block k: [pair_indptr[k], pair_indptr[k+1])
 *   S[...]                                    block order; nnz_d values for diagonal blocks,
 *                                             nnz_o for off-diagonal blocks, pattern order
 *   U[n_pairs*b], V[n_pairs*b]                one row of b values per pair
 *   x, y[nc*b]                                cell-major vectors
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC oracle.c -o liboracle.so
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef long long i64;

/* Start of each block's S values: diagonal blocks hold nnz_d values, the others nnz_o. */
static i64 *block_offsets(int nc, const int *block_indptr, const int *block_indices,
                          int nnz_d, int nnz_o)
{
    int nnzb = block_indptr[nc];
    i64 *off = (i64 *)malloc(sizeof(i64) * (size_t)(nnzb + 1));
    off[0] = 0;
    for (int i = 0; i < nc; i++)
        for (int k = block_indptr[i]; k < block_indptr[i + 1]; k++)
            off[k + 1] = off[k] + (block_indices[k] == i ? nnz_d : nnz_o);
    return off;
}

/* D = S (scattered from its CSR pattern) + sum over the block's pairs of u v^T. */
static void assemble_block(int b, const int *indptr, const int *indices, const double *s,
                           int p0, int p1, const double *U, const double *V, double *D)
{
    memset(D, 0, sizeof(double) * (size_t)b * b);
    for (int p = 0; p < b; p++)
        for (int e = indptr[p]; e < indptr[p + 1]; e++)
            D[(size_t)p * b + indices[e]] = s[e];
    for (int k = p0; k < p1; k++) {
        const double *u = U + (size_t)k * b, *v = V + (size_t)k * b;
        for (int p = 0; p < b; p++)
            for (int q = 0; q < b; q++)
                D[(size_t)p * b + q] += u[p] * v[q];
    }
}

/* Assemble stored block k (block row i) into D. */
static void assemble_stored_block(int i, int k, int b, const int *block_indices,
                                  const int *d_indptr, const int *d_indices,
                                  const int *o_indptr, const int *o_indices,
                                  const int *pair_indptr, const i64 *soff,
                                  const double *S, const double *U, const double *V,
                                  double *D)
{
    int diag = block_indices[k] == i;
    assemble_block(b, diag ? d_indptr : o_indptr, diag ? d_indices : o_indices,
                   S + soff[k], pair_indptr[k], pair_indptr[k + 1], U, V, D);
}

/* Column view of the block structure: for every column cell j, the (row, block) pairs. */
static void block_transpose(int nc, const int *block_indptr, const int *block_indices,
                            int *col_ptr, int *col_row, int *col_blk)
{
    int nnzb = block_indptr[nc];
    memset(col_ptr, 0, sizeof(int) * (size_t)(nc + 1));
    for (int k = 0; k < nnzb; k++) col_ptr[block_indices[k] + 1]++;
    for (int j = 0; j < nc; j++) col_ptr[j + 1] += col_ptr[j];
    int *fill = (int *)malloc(sizeof(int) * (size_t)nc);
    memcpy(fill, col_ptr, sizeof(int) * (size_t)nc);
    for (int i = 0; i < nc; i++)
        for (int k = block_indptr[i]; k < block_indptr[i + 1]; k++) {
            int j = block_indices[k], t = fill[j]++;
            col_row[t] = i;
            col_blk[t] = k;
        }
    free(fill);
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* y = D x (trans = 0) or y = D^T x (trans = 1), D assembled block by block. */
void orc_matvec(int nc, int b, const int *block_indptr, const int *block_indices,
                const int *d_indptr, const int *d_indices, const int *o_indptr,
                const int *o_indices, const int *pair_indptr, const double *S,
                const double *U, const double *V, const double *x, double *y, int trans)
{
    int nnz_d = d_indptr[b], nnz_o = o_indptr[b];
    i64 *soff = block_offsets(nc, block_indptr, block_indices, nnz_d, nnz_o);
    int nnzb = block_indptr[nc];
    int *col_ptr = NULL, *col_row = NULL, *col_blk = NULL;
    if (trans) {
        col_ptr = (int *)malloc(sizeof(int) * (size_t)(nc + 1));
        col_row = (int *)malloc(sizeof(int) * (size_t)nnzb);
        col_blk = (int *)malloc(sizeof(int) * (size_t)nnzb);
        block_transpose(nc, block_indptr, block_indices, col_ptr, col_row, col_blk);
    }
#pragma omp parallel
    {
        double *D = (double *)malloc(sizeof(double) * (size_t)b * b);
#pragma omp for schedule(static)
        for (int c = 0; c < nc; c++) {
            double *yc = y + (size_t)c * b;
            for (int p = 0; p < b; p++) yc[p] = 0.0;
            if (!trans) {
                /* row c: y_c = sum_j D_cj x_j */
                for (int k = block_indptr[c]; k < block_indptr[c + 1]; k++) {
                    int j = block_indices[k];
                    assemble_stored_block(c, k, b, block_indices, d_indptr, d_indices, o_indptr,
                                          o_indices, pair_indptr, soff, S, U, V, D);
                    const double *xj = x + (size_t)j * b;
                    for (int p = 0; p < b; p++) {
                        double acc = 0.0;
                        for (int q = 0; q < b; q++) acc += D[(size_t)p * b + q] * xj[q];
                        yc[p] += acc;
                    }
                }
            } else {
                /* column c: y_c = sum_i D_ic^T x_i */
                for (int t = col_ptr[c]; t < col_ptr[c + 1]; t++) {
                    int i = col_row[t], k = col_blk[t];
                    assemble_stored_block(i, k, b, block_indices, d_indptr, d_indices, o_indptr,
                                          o_indices, pair_indptr, soff, S, U, V, D);
                    const double *xi = x + (size_t)i * b;
                    for (int q = 0; q < b; q++) {
                        double acc = 0.0;
                        for (int p = 0; p < b; p++) acc += D[(size_t)p * b + q] * xi[p];
                        yc[q] += acc;
                    }
                }
            }
        }
        free(D);
    }
    free(soff);
    free(col_ptr);
    free(col_row);
    free(col_blk);
}

/* Selected entries of y = D x (or D^T x): out[s] = y[rows[s]], rows[s] = cell*b + component. */
void orc_matvec_rows(int nc, int b, const int *block_indptr, const int *block_indices,
                     const int *d_indptr, const int *d_indices, const int *o_indptr,
                     const int *o_indices, const int *pair_indptr, const double *S,
                     const double *U, const double *V, const double *x, int trans,
                     int n_rows, const i64 *rows, double *out)
{
    int nnz_d = d_indptr[b], nnz_o = o_indptr[b];
    i64 *soff = block_offsets(nc, block_indptr, block_indices, nnz_d, nnz_o);
    int nnzb = block_indptr[nc];
    int *col_ptr = (int *)malloc(sizeof(int) * (size_t)(nc + 1));
    int *col_row = (int *)malloc(sizeof(int) * (size_t)nnzb);
    int *col_blk = (int *)malloc(sizeof(int) * (size_t)nnzb);
    block_transpose(nc, block_indptr, block_indices, col_ptr, col_row, col_blk);
#pragma omp parallel
    {
        double *D = (double *)malloc(sizeof(double) * (size_t)b * b);
#pragma omp for schedule(dynamic, 16)
        for (int s = 0; s < n_rows; s++) {
            int c = (int)(rows[s] / b), p = (int)(rows[s] % b);
            double acc = 0.0;
            if (!trans) {
                for (int k = block_indptr[c]; k < block_indptr[c + 1]; k++) {
                    const double *xj = x + (size_t)block_indices[k] * b;
                    assemble_stored_block(c, k, b, block_indices, d_indptr, d_indices, o_indptr,
                                          o_indices, pair_indptr, soff, S, U, V, D);
                    for (int q = 0; q < b; q++) acc += D[(size_t)p * b + q] * xj[q];
                }
            } else {
                for (int t = col_ptr[c]; t < col_ptr[c + 1]; t++) {
                    int i = col_row[t], k = col_blk[t];
                    const double *xi = x + (size_t)i * b;
                    assemble_stored_block(i, k, b, block_indices, d_indptr, d_indices, o_indptr,
                                          o_indices, pair_indptr, soff, S, U, V, D);
                    for (int q = 0; q < b; q++) acc += D[(size_t)q * b + p] * xi[q];
                }
            }
            out[s] = acc;
        }
        free(D);
    }
    free(soff);
    free(col_ptr);
    free(col_row);
    free(col_blk);
}

/* Textbook LU with partial pivoting, in place: P A = L U, L unit lower.
 * piv[k] = row swapped with row k at step k.  Returns 0, or 1 on a zero pivot. */
static int lu_factor(int b, double *A, int *piv)
{
    for (int k = 0; k < b; k++) {
        int r = k;
        double best = fabs(A[(size_t)k * b + k]);
        for (int i = k + 1; i < b; i++)
            if (fabs(A[(size_t)i * b + k]) > best) {
                best = fabs(A[(size_t)i * b + k]);
                r = i;
            }
        piv[k] = r;
        if (best == 0.0) return 1;
        if (r != k)
            for (int j = 0; j < b; j++) {
                double t = A[(size_t)k * b + j];
                A[(size_t)k * b + j] = A[(size_t)r * b + j];
                A[(size_t)r * b + j] = t;
            }
        for (int i = k + 1; i < b; i++) {
            double l = A[(size_t)i * b + k] / A[(size_t)k * b + k];
            A[(size_t)i * b + k] = l;
            for (int j = k + 1; j < b; j++) A[(size_t)i * b + j] -= l * A[(size_t)k * b + j];
        }
    }
    return 0;
}

/* Solve A z = x (trans = 0) or A^T z = x (trans = 1) from the factors of lu_factor. */
static void lu_solve(int b, const double *LU, const int *piv, const double *x, double *z,
                     int trans)
{
    for (int p = 0; p < b; p++) z[p] = x[p];
    if (!trans) {
        for (int k = 0; k < b; k++)
            if (piv[k] != k) {
                double t = z[k];
                z[k] = z[piv[k]];
                z[piv[k]] = t;
            }
        for (int i = 0; i < b; i++)          /* L w = P x, unit diagonal */
            for (int j = 0; j < i; j++) z[i] -= LU[(size_t)i * b + j] * z[j];
        for (int i = b - 1; i >= 0; i--) {  /* U z = w */
            for (int j = i + 1; j < b; j++) z[i] -= LU[(size_t)i * b + j] * z[j];
            z[i] /= LU[(size_t)i * b + i];
        }
    } else {
        /* A^T = U^T L^T P: U^T w = x, L^T v = w, z = P^T v */
        for (int i = 0; i < b; i++) {
            for (int j = 0; j < i; j++) z[i] -= LU[(size_t)j * b + i] * z[j];
            z[i] /= LU[(size_t)i * b + i];
        }
        for (int i = b - 1; i >= 0; i--)
            for (int j = i + 1; j < b; j++) z[i] -= LU[(size_t)j * b + i] * z[j];
        for (int k = b - 1; k >= 0; k--)
            if (piv[k] != k) {
                double t = z[k];
                z[k] = z[piv[k]];
                z[piv[k]] = t;
            }
    }
}

/* Factor every diagonal block D_ii.  LU[nc*b*b], piv[nc*b].
 * Returns 0, or -(1 + cell) for the first cell whose block is singular. */
int orc_bj_setup(int nc, int b, const int *block_indptr, const int *block_indices,
                 const int *d_indptr, const int *d_indices, const int *o_indptr,
                 const int *o_indices, const int *pair_indptr, const double *S,
                 const double *U, const double *V, double *LU, int *piv)
{
    int nnz_d = d_indptr[b], nnz_o = o_indptr[b];
    i64 *soff = block_offsets(nc, block_indptr, block_indices, nnz_d, nnz_o);
    int bad = nc;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < nc; c++) {
        int kd = -1;
        for (int k = block_indptr[c]; k < block_indptr[c + 1]; k++)
            if (block_indices[k] == c) kd = k;
        double *A = LU + (size_t)c * b * b;
        int err = 1;
        if (kd >= 0) {
            assemble_stored_block(c, kd, b, block_indices, d_indptr, d_indices, o_indptr,
                                  o_indices, pair_indptr, soff, S, U, V, A);
            err = lu_factor(b, A, piv + (size_t)c * b);
        }
        if (err) {
#pragma omp critical
            if (c < bad) bad = c;
        }
    }
    free(soff);
    return bad < nc ? -(1 + bad) : 0;
}

/* z_i = D_ii^-1 x_i (trans = 0) or D_ii^-T x_i (trans = 1) for every cell. */
void orc_bj_apply(int nc, int b, const double *LU, const int *piv, const double *x,
                  double *z, int trans)
{
#pragma omp parallel for schedule(static)
    for (int c = 0; c < nc; c++)
        lu_solve(b, LU + (size_t)c * b * b, piv + (size_t)c * b, x + (size_t)c * b,
                 z + (size_t)c * b, trans);
}

/* Block-Jacobi on a subset of cells (factor + solve each): out[s*b..] = D_cc^-1 x_c.
 * Returns 0, or -(1 + s) for the first sampled cell whose block is singular. */
int orc_bj_cells(int nc, int b, const int *block_indptr, const int *block_indices,
                 const int *d_indptr, const int *d_indices, const int *o_indptr,
                 const int *o_indices, const int *pair_indptr, const double *S,
                 const double *U, const double *V, const double *x, int trans,
                 int n_sample, const int *cells, double *out)
{
    int nnz_d = d_indptr[b], nnz_o = o_indptr[b];
    i64 *soff = block_offsets(nc, block_indptr, block_indices, nnz_d, nnz_o);
    int bad = n_sample;
#pragma omp parallel
    {
        double *A = (double *)malloc(sizeof(double) * (size_t)b * b);
        int *pv = (int *)malloc(sizeof(int) * (size_t)b);
#pragma omp for schedule(dynamic, 4)
        for (int s = 0; s < n_sample; s++) {
            int c = cells[s], kd = -1;
            for (int k = block_indptr[c]; k < block_indptr[c + 1]; k++)
                if (block_indices[k] == c) kd = k;
            int err = 1;
            if (kd >= 0) {
                assemble_stored_block(c, kd, b, block_indices, d_indptr, d_indices, o_indptr,
                                      o_indices, pair_indptr, soff, S, U, V, A);
                err = lu_factor(b, A, pv);
            }
            if (err) {
#pragma omp critical
                if (s < bad) bad = s;
            } else {
                lu_solve(b, A, pv, x + (size_t)c * b, out + (size_t)s * b, trans);
            }
        }
        free(A);
        free(pv);
    }
    free(soff);
    return bad < n_sample ? -(1 + bad) : 0;
}

/* Adjoint outer products of x = J^-1 b for the cotangent lambda = J^-T g:
 *   gS[block (i,j)][entry (p,q)] = -lambda_i[p] x_j[q]
 *   gU[pair of (i,j)] = -(v . x_j) lambda_i,   gV[pair of (i,j)] = -(u . lambda_i) x_j  */
void orc_grad(int nc, int b, const int *block_indptr, const int *block_indices,
              const int *d_indptr, const int *d_indices, const int *o_indptr,
              const int *o_indices, const int *pair_indptr, const double *U,
              const double *V, const double *lambda, const double *x, double *gS,
              double *gU, double *gV)
{
    int nnz_d = d_indptr[b], nnz_o = o_indptr[b];
    i64 *soff = block_offsets(nc, block_indptr, block_indices, nnz_d, nnz_o);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nc; i++) {
        const double *li = lambda + (size_t)i * b;
        for (int k = block_indptr[i]; k < block_indptr[i + 1]; k++) {
            int j = block_indices[k];
            const double *xj = x + (size_t)j * b;
            const int *ip = j == i ? d_indptr : o_indptr;
            const int *ix = j == i ? d_indices : o_indices;
            double *g = gS + soff[k];
            for (int p = 0; p < b; p++)
                for (int e = ip[p]; e < ip[p + 1]; e++) g[e] = -li[p] * xj[ix[e]];
            for (int t = pair_indptr[k]; t < pair_indptr[k + 1]; t++) {
                const double *u = U + (size_t)t * b, *v = V + (size_t)t * b;
                double vx = 0.0, ul = 0.0;
                for (int q = 0; q < b; q++) vx += v[q] * xj[q];
                for (int p = 0; p < b; p++) ul += u[p] * li[p];
                for (int p = 0; p < b; p++) gU[(size_t)t * b + p] = -vx * li[p];
                for (int q = 0; q < b; q++) gV[(size_t)t * b + q] = -ul * xj[q];
            }
        }
    }
    free(soff);
}
