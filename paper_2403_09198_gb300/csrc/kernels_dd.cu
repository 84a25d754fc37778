// kernels_dd.cu -- domain decomposition of the hot path: sub-domain plans, the
// halo exchange of the matvec, and restarted GMRES over several parts.
//
// The block adjacency of Section 5.1 couples a cell with its face neighbours
// only, and the block-Jacobi preconditioner of Section 6 is one block per cell,
// so the work shards by cells.  Each part is an ordinary square handle over its
// owned cells followed by its ghost cells (see sts.h); one halo exchange before
// every matvec fills the ghost entries of the input, after which the local
// product is exact at the owned rows in both directions.  GMRES runs the same
// steps as the single-handle solver (kernels_krylov.cu), with the dot products
// of each part summed on the host over the parts of this process and then over
// the processes by the caller's allreduce.
//
// The driver (dd_gmres) is written against an interface of vector operations
// named by index, with two implementations: the library's kernels on the parts
// of this process (GpuOps), and operations supplied through the C ABI (CbOps,
// sts_dd_gmres_ops), which is how its control flow runs on CPU ranks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "sts_internal.h"

struct sts_dd_plan_s {
    int n_cells = 0, n_parts = 0, part = 0, n_owned = 0;
    std::vector<int> gptr, gidx;        // global block CSR (for block kinds and value offsets)
    std::vector<int> l2g;               // owned (ascending global id), then ghosts (ascending)
    std::vector<int> bptr, bidx, bmap;  // local block CSR and the global block of each local block
    std::vector<int> nbr, send_ptr, send_cells, recv_ptr, recv_cells;
};

namespace sts {
namespace {

sts_status plan_create(int nc, const int *bptr, const int *bidx, int n_parts, const int *part_of, int part,
                       sts_dd_plan_s **out) {
    if (nc < 1 || !bptr || !bidx || !part_of || n_parts < 1 || part < 0 || part >= n_parts)
        return set_error(STS_ERR_INVALID_ARG, "sts_dd_plan_create: bad sizes or NULL array");
    if (bptr[0] != 0) return set_error(STS_ERR_INVALID_ARG, "sts_dd_plan_create: block_indptr[0] must be 0");
    for (int i = 0; i < nc; ++i) {
        if (bptr[i + 1] < bptr[i]) return set_error(STS_ERR_INVALID_ARG, "sts_dd_plan_create: indptr decreases");
        bool diag = false;
        for (int k = bptr[i]; k < bptr[i + 1]; ++k) {
            if (bidx[k] < 0 || bidx[k] >= nc || (k > bptr[i] && bidx[k] <= bidx[k - 1]))
                return set_error(STS_ERR_INVALID_ARG, "sts_dd_plan_create: block row %d not sorted or out of range", i);
            diag = diag || bidx[k] == i;
        }
        if (!diag) return set_error(STS_ERR_INVALID_ARG, "sts_dd_plan_create: block row %d has no diagonal", i);
        if (part_of[i] < 0 || part_of[i] >= n_parts)
            return set_error(STS_ERR_INVALID_ARG, "sts_dd_plan_create: part_of_cell[%d] = %d out of range", i,
                             part_of[i]);
    }
    auto P = new sts_dd_plan_s();
    P->n_cells = nc;
    P->n_parts = n_parts;
    P->part = part;
    const int nnzb = bptr[nc];
    P->gptr.assign(bptr, bptr + nc + 1);
    P->gidx.assign(bidx, bidx + nnzb);
    // column adjacency (who has a block in my column)
    std::vector<int> cptr(nc + 1, 0), crow(nnzb);
    for (int k = 0; k < nnzb; ++k) cptr[bidx[k] + 1]++;
    for (int c = 0; c < nc; ++c) cptr[c + 1] += cptr[c];
    {
        std::vector<int> fill(cptr.begin(), cptr.end() - 1);
        for (int i = 0; i < nc; ++i)
            for (int k = bptr[i]; k < bptr[i + 1]; ++k) crow[fill[bidx[k]]++] = i;
    }
    std::vector<int> g2l(nc, -1);
    for (int c = 0; c < nc; ++c)
        if (part_of[c] == part) {
            g2l[c] = (int)P->l2g.size();
            P->l2g.push_back(c);
        }
    P->n_owned = (int)P->l2g.size();
    if (P->n_owned == 0) {
        delete P;
        return set_error(STS_ERR_INVALID_ARG, "sts_dd_plan_create: part %d owns no cell", part);
    }
    // ghosts: cells of other parts sharing a block with an owned cell, either direction
    std::vector<char> is_ghost(nc, 0);
    std::vector<std::vector<int>> send_to(n_parts);     // owned local ids per destination part
    for (int li = 0; li < P->n_owned; ++li) {
        const int i = P->l2g[li];
        std::vector<int> dest;
        auto touch = [&](int j) {
            if (part_of[j] == part) return;
            is_ghost[j] = 1;
            dest.push_back(part_of[j]);
        };
        for (int k = bptr[i]; k < bptr[i + 1]; ++k) touch(bidx[k]);
        for (int k = cptr[i]; k < cptr[i + 1]; ++k) touch(crow[k]);
        std::sort(dest.begin(), dest.end());
        dest.erase(std::unique(dest.begin(), dest.end()), dest.end());
        for (int q : dest) send_to[q].push_back(li);
    }
    for (int c = 0; c < nc; ++c)
        if (is_ghost[c]) {
            g2l[c] = (int)P->l2g.size();
            P->l2g.push_back(c);
        }
    const int nl = (int)P->l2g.size();
    // local block rows: owned rows keep every block, ghost rows their diagonal and
    // their blocks into owned columns; columns ascending by local id
    P->bptr.assign(1, 0);
    for (int li = 0; li < nl; ++li) {
        const int i = P->l2g[li];
        std::vector<std::pair<int, int>> row;      // (local column, global block)
        for (int k = bptr[i]; k < bptr[i + 1]; ++k) {
            const int lj = g2l[bidx[k]];
            if (li < P->n_owned) {
                if (lj < 0) {
                    delete P;
                    return set_error(STS_ERR_INVALID_ARG, "sts_dd_plan_create: internal: column outside the sub-domain");
                }
                row.push_back({lj, k});
            } else if (bidx[k] == i || (lj >= 0 && lj < P->n_owned)) {
                row.push_back({lj, k});
            }
        }
        std::sort(row.begin(), row.end());
        for (auto &e : row) {
            P->bidx.push_back(e.first);
            P->bmap.push_back(e.second);
        }
        P->bptr.push_back((int)P->bidx.size());
    }
    // exchange lists: ghosts grouped by owner part, each in ascending global id
    std::vector<std::vector<int>> recv_from(n_parts);
    for (int li = P->n_owned; li < nl; ++li) recv_from[part_of[P->l2g[li]]].push_back(li);
    P->send_ptr.assign(1, 0);
    P->recv_ptr.assign(1, 0);
    for (int q = 0; q < n_parts; ++q) {
        if (q == part || (send_to[q].empty() && recv_from[q].empty())) continue;
        P->nbr.push_back(q);
        P->send_cells.insert(P->send_cells.end(), send_to[q].begin(), send_to[q].end());
        P->recv_cells.insert(P->recv_cells.end(), recv_from[q].begin(), recv_from[q].end());
        P->send_ptr.push_back((int)P->send_cells.size());
        P->recv_ptr.push_back((int)P->recv_cells.size());
    }
    *out = P;
    return STS_OK;
}

// pairs of every global block: from pair_indptr or the uniform counts
std::vector<long long> global_pair_base(const sts_dd_plan_s *P, const int *pair_indptr, int r_diag, int r_off) {
    const int nnzb = P->gptr[P->n_cells];
    std::vector<long long> pb(nnzb + 1, 0);
    for (int i = 0; i < P->n_cells; ++i)
        for (int k = P->gptr[i]; k < P->gptr[i + 1]; ++k)
            pb[k + 1] = pair_indptr ? pair_indptr[k + 1] : pb[k] + (P->gidx[k] == i ? r_diag : r_off);
    return pb;
}

std::vector<long long> global_s_base(const sts_dd_plan_s *P, int nnz_d, int nnz_o) {
    const int nnzb = P->gptr[P->n_cells];
    std::vector<long long> sb(nnzb + 1, 0);
    for (int i = 0; i < P->n_cells; ++i)
        for (int k = P->gptr[i]; k < P->gptr[i + 1]; ++k) sb[k + 1] = sb[k] + (P->gidx[k] == i ? nnz_d : nnz_o);
    return sb;
}

// One warp per segment: dst[dst_off[s] + e] = src[src_off[s] + e], e < len[s].
__global__ void k_gather_segments(double *dst, const double *src, const long long *src_off,
                                  const long long *dst_off, const int *len, int nseg) {
    const int lane = threadIdx.x & 31;
    for (long long s = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < nseg;
         s += (long long)gridDim.x * (blockDim.x >> 5)) {
        const double *a = src + src_off[s];
        double *b = dst + dst_off[s];
        for (int e = lane; e < len[s]; e += 32) b[e] = a[e];
    }
}

// Halo kernels on internal vectors [b][ncp] (component-major).
// copy: dst[q][dc[i]] = src[q][sc[i]]; pack: buf[i][q] = src[q][sc[i]];
// unpack: dst[q][dc[i]] = buf[i][q].
__global__ void k_halo_copy(double *dst, int ncp_d, const int *dc, const double *src, int ncp_s, const int *sc, int n,
                            int b) {
    const long long total = (long long)n * b;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(e / n), i = (int)(e - (long long)q * n);
        dst[(size_t)q * ncp_d + dc[i]] = src[(size_t)q * ncp_s + sc[i]];
    }
}

__global__ void k_halo_pack(double *buf, const double *src, int ncp, const int *sc, int n, int b) {
    const long long total = (long long)n * b;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / b), q = (int)(e - (long long)i * b);
        buf[e] = src[(size_t)q * ncp + sc[i]];
    }
}

__global__ void k_halo_unpack(double *dst, int ncp, const int *dc, const double *buf, int n, int b) {
    const long long total = (long long)n * b;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / b), q = (int)(e - (long long)i * b);
        dst[(size_t)q * ncp + dc[i]] = buf[e];
    }
}

// Zero the entries of cells c >= c0 (ghost and padding cells) of an internal vector.
__global__ void k_zero_cells(double *x, int ncp, int c0, int b) {
    const int w = ncp - c0;
    const long long total = (long long)w * b;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(e / w), c = c0 + (int)(e - (long long)q * w);
        x[(size_t)q * ncp + c] = 0.0;
    }
}

inline int grid_of(long long n) {
    long long g = (n + 255) / 256;
    return (int)std::max(1LL, std::min(g, 152LL * 16));
}

// ---------------------------------------------------------------------------
// The driver.  Vector indices: 0..m basis, m+1..2m preconditioned vectors,
// 2m+1 w, 2m+2 r, 2m+3 x, 2m+4 b.
struct DdOps {
    virtual ~DdOps() {}
    virtual sts_status matvec(int in, int out) = 0;
    virtual sts_status apply(int in, int out) = 0;
    virtual sts_status copy(int out, int in) = 0;
    virtual sts_status sub(int out, int a, int b) = 0;
    virtual sts_status scale(int out, int in, double s) = 0;
    virtual sts_status dots(int v0, int k, int w, int self, double *out) = 0;
    virtual sts_status update(int w, int v0, int k, const double *h, int norm, double *out) = 0;
    virtual sts_status norm2(int v, double *out) = 0;
    virtual sts_status axpy(int x, int v0, int k, const double *y) = 0;
    virtual sts_status allreduce(double *vals, int n) = 0;
};

struct DdParams {
    int m = 30, max_iters = 1000;
    double rtol = 1e-10;
    bool pre = true;
    double *history = nullptr;
};

sts_status dd_options(const sts_gmres_opts *o, bool need_setup_ok, DdParams *P, int *dir) {
    sts_gmres_opts d{};
    if (o) d = *o;
    if (d.left || d.mixed) return set_error(STS_ERR_INVALID_ARG, "dd gmres: left and mixed modes are not supported");
    if (d.precond != STS_PRECOND_BJ && d.precond != STS_PRECOND_NONE)
        return set_error(STS_ERR_INVALID_ARG, "dd gmres: unknown precond %d", d.precond);
    P->m = d.restart > 0 ? d.restart : 30;
    if (P->m > 512) return set_error(STS_ERR_INVALID_ARG, "dd gmres: restart %d exceeds 512", P->m);
    P->max_iters = d.max_iters > 0 ? d.max_iters : 1000;
    P->rtol = d.rtol > 0 ? d.rtol : 1e-10;
    P->pre = d.precond != STS_PRECOND_NONE;
    P->history = d.history;
    *dir = d.trans ? 1 : 0;
    (void)need_setup_ok;
    return STS_OK;
}

sts_status dd_gmres(DdOps &ops, const DdParams &P, sts_gmres_info *info) {
    const int m = P.m;
    const int VW = 2 * m + 1, VR = 2 * m + 2, VX = 2 * m + 3, VB = 2 * m + 4;
    auto Zi = [&](int j) { return m + 1 + j; };
    // ||b||^2 and ||x0||^2 in one sum: a zero guess starts from r = b without a product
    double t[2];
    STS_TRY(ops.norm2(VB, t));
    STS_TRY(ops.norm2(VX, t + 1));
    STS_TRY(ops.allreduce(t, 2));
    const double bnorm = std::sqrt(t[0]);
    bool zero_guess = t[1] == 0.0;
    if (!std::isfinite(bnorm)) return set_error(STS_ERR_NUMERIC, "dd gmres: right-hand side has NaN or Inf");
    sts_gmres_info inf{0, 0, 1, 0.0, 0, 0};
    sts_status status = STS_OK;
    if (bnorm == 0.0) {
        STS_TRY(ops.scale(VX, VX, 0.0));
    } else {
        std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m), h1(m + 2), h2(m + 2);
        int its = 0;
        for (;;) {
            NvtxRange nvtx_cycle("dd gmres cycle");
            double beta = bnorm;
            if (zero_guess) {
                STS_TRY(ops.copy(VR, VB));
                zero_guess = false;
            } else {
                STS_TRY(ops.matvec(VX, VW));
                ++inf.matvecs;
                STS_TRY(ops.sub(VR, VB, VW));
                STS_TRY(ops.norm2(VR, t));
                STS_TRY(ops.allreduce(t, 1));
                beta = std::sqrt(t[0]);
            }
            if (!std::isfinite(beta)) {
                status = set_error(STS_ERR_NUMERIC, "dd gmres: residual norm is NaN or Inf");
                break;
            }
            inf.true_rel_residual = beta / bnorm;
            if (beta / bnorm <= P.rtol) { inf.converged = 1; break; }
            if (its >= P.max_iters) { inf.converged = 0; break; }
            const double stop_abs = P.rtol * bnorm;
            STS_TRY(ops.scale(0, VR, 1.0 / beta));
            std::fill(g.begin(), g.end(), 0.0);
            g[0] = beta;
            int k = 0;
            for (int j = 0; j < m; ++j) {
                NvtxRange nvtx_step("dd gmres arnoldi step");
                if (P.pre) STS_TRY(ops.apply(j, Zi(j)));
                else STS_TRY(ops.copy(Zi(j), j));
                STS_TRY(ops.matvec(Zi(j), VW));
                ++inf.matvecs;
                if (P.pre) ++inf.applies;
                // CGS2: h1 = V^T w (+ w.w), w -= V h1; h2 = V^T w, w -= V h2, ||w||^2
                STS_TRY(ops.dots(0, j + 1, VW, 1, h1.data()));
                STS_TRY(ops.allreduce(h1.data(), j + 2));
                STS_TRY(ops.update(VW, 0, j + 1, h1.data(), 0, nullptr));
                STS_TRY(ops.dots(0, j + 1, VW, 0, h2.data()));
                STS_TRY(ops.allreduce(h2.data(), j + 1));
                STS_TRY(ops.update(VW, 0, j + 1, h2.data(), 1, t));
                STS_TRY(ops.allreduce(t, 1));
                const double w0 = std::sqrt(h1[j + 1]);
                const double hn = std::sqrt(t[0]);
                bool bad = !std::isfinite(w0) || !std::isfinite(hn);
                for (int i = 0; i <= j; ++i) {
                    H[(size_t)i * m + j] = h1[i] + h2[i];
                    bad = bad || !std::isfinite(H[(size_t)i * m + j]);
                }
                if (bad) { status = set_error(STS_ERR_NUMERIC, "dd gmres: NaN or Inf in the Arnoldi process"); break; }
                H[(size_t)(j + 1) * m + j] = hn;
                for (int i = 0; i < j; ++i) {
                    const double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
                    H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
                    H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
                }
                const double hjj = H[(size_t)j * m + j];
                const double den = std::hypot(hjj, hn);
                cs[j] = hjj / den;
                sn[j] = hn / den;
                H[(size_t)j * m + j] = den;
                H[(size_t)(j + 1) * m + j] = 0.0;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                ++its;
                k = j + 1;
                if (P.history && its <= P.max_iters) P.history[its - 1] = std::fabs(g[j + 1]) * (1.0 / bnorm);
                const bool happy = hn <= 1e-14 * w0;
                if (happy || std::fabs(g[j + 1]) <= stop_abs || its >= P.max_iters) break;
                STS_TRY(ops.scale(j + 1, VW, 1.0 / hn));
            }
            if (status != STS_OK) break;
            for (int i = k - 1; i >= 0; --i) {
                double s = g[i];
                for (int l = i + 1; l < k; ++l) s -= H[(size_t)i * m + l] * y[l];
                y[i] = s / H[(size_t)i * m + i];
            }
            STS_TRY(ops.axpy(VX, Zi(0), k, y.data()));
            ++inf.restarts;
        }
        inf.iterations = its;
    }
    if (info) *info = inf;
    if (status != STS_OK) return status;
    if (!inf.converged)
        return set_error(STS_ERR_NOT_CONVERGED, "dd gmres: %d iterations, true relative residual %.3e > rtol %.3e",
                         inf.iterations, inf.true_rel_residual, P.rtol);
    return STS_OK;
}

// Operations supplied by the caller (sts_dd_gmres_ops).
struct CbOps final : DdOps {
    const sts_dd_ops *o;
    explicit CbOps(const sts_dd_ops *o_) : o(o_) {}
    static sts_status st(int rc, const char *what) {
        return rc == 0 ? STS_OK : set_error(STS_ERR_COMM, "sts_dd_gmres_ops: the %s callback returned %d", what, rc);
    }
    sts_status matvec(int in, int out) override { return st(o->matvec(o->ctx, in, out), "matvec"); }
    sts_status apply(int in, int out) override { return st(o->apply(o->ctx, in, out), "apply"); }
    sts_status copy(int out, int in) override { return st(o->copy(o->ctx, out, in), "copy"); }
    sts_status sub(int out, int a, int b) override { return st(o->sub(o->ctx, out, a, b), "sub"); }
    sts_status scale(int out, int in, double s) override { return st(o->scale(o->ctx, out, in, s), "scale"); }
    sts_status dots(int v0, int k, int w, int self, double *out) override {
        return st(o->dots(o->ctx, v0, k, w, self, out), "dots");
    }
    sts_status update(int w, int v0, int k, const double *h, int norm, double *out) override {
        return st(o->update(o->ctx, w, v0, k, h, norm, out), "update");
    }
    sts_status norm2(int v, double *out) override { return st(o->norm2(o->ctx, v, out), "norm2"); }
    sts_status axpy(int x, int v0, int k, const double *y) override { return st(o->axpy(o->ctx, x, v0, k, y), "axpy"); }
    sts_status allreduce(double *vals, int n) override { return st(o->allreduce(o->ctx, vals, n), "allreduce"); }
};

}  // namespace
}  // namespace sts

// ---------------------------------------------------------------------------
// Parts of this process on the GPU.
struct sts_dd_s {
    struct Link {
        int peer = -1;            // neighbour part id
        int local_peer = -1;      // its index among this process's parts, or -1 (another process)
        int n_send = 0, n_recv = 0;
        int *d_send = nullptr;    // owned local cells sent to the peer
        int *d_recv = nullptr;    // ghost local cells received from the peer
        int *d_peer_send = nullptr;   // in-process peer: its send list to this part (alias)
        double *sbuf = nullptr, *rbuf = nullptr;   // messages to / from another process
    };
    std::vector<sts_jac_s *> jac;
    std::vector<sts_dd_plan_s *> plan;
    std::vector<int> part_ids;
    std::vector<std::vector<Link>> links;
    bool has_comm = false;
    sts_dd_comm comm{};
    cudaStream_t stream = nullptr;
    int b = 0;
    std::vector<void *> owned;    // device allocations of this object
};

namespace sts {
namespace {

sts_status dd_alloc(sts_dd_s *d, void **p, size_t bytes) {
    *p = nullptr;
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(STS_ERR_ALLOC, "sts_dd_create: cudaMalloc of %zu bytes failed: %s", bytes,
                         cudaGetErrorString(e));
    }
    d->owned.push_back(*p);
    return STS_OK;
}

void dd_free(sts_dd_s *d) {
    for (void *p : d->owned) cudaFree(p);
    d->owned.clear();
}

// Fill the ghost entries of dst[p] (internal vectors) from the owned entries of
// src[q] of the neighbouring parts: in-process neighbours by one copy kernel,
// the others through the caller's exchange.
sts_status halo(sts_dd_s *d, const std::vector<const double *> &src, const std::vector<double *> &dst) {
    const int np = (int)d->jac.size(), b = d->b;
    std::vector<int> s_from, s_to, s_len, r_from, r_to, r_len;
    std::vector<const double *> s_buf;
    std::vector<double *> r_buf;
    for (int p = 0; p < np; ++p) {
        sts_jac_s *h = d->jac[p];
        for (auto &L : d->links[p]) {
            if (L.local_peer >= 0) {
                if (L.n_recv == 0) continue;
                sts_jac_s *hq = d->jac[L.local_peer];
                k_halo_copy<<<grid_of((long long)L.n_recv * b), 256, 0, d->stream>>>(
                    dst[p], h->ncp, L.d_recv, src[L.local_peer], hq->ncp, L.d_peer_send, L.n_recv, b);
                STS_LAUNCHED();
            } else {
                if (L.n_send > 0) {
                    k_halo_pack<<<grid_of((long long)L.n_send * b), 256, 0, d->stream>>>(L.sbuf, src[p], h->ncp,
                                                                                          L.d_send, L.n_send, b);
                    STS_LAUNCHED();
                    s_from.push_back(d->part_ids[p]);
                    s_to.push_back(L.peer);
                    s_buf.push_back(L.sbuf);
                    s_len.push_back(L.n_send * b);
                }
                if (L.n_recv > 0) {
                    r_from.push_back(L.peer);
                    r_to.push_back(d->part_ids[p]);
                    r_buf.push_back(L.rbuf);
                    r_len.push_back(L.n_recv * b);
                }
            }
        }
    }
    if (s_buf.empty() && r_buf.empty()) return STS_OK;
    const int rc = d->comm.exchange(d->comm.ctx, (int)s_buf.size(), s_from.data(), s_to.data(), s_buf.data(),
                                    s_len.data(), (int)r_buf.size(), r_from.data(), r_to.data(), r_buf.data(),
                                    r_len.data(), d->stream);
    if (rc != 0) return set_error(STS_ERR_COMM, "dd halo exchange: the exchange callback returned %d", rc);
    for (int p = 0; p < np; ++p)
        for (auto &L : d->links[p])
            if (L.local_peer < 0 && L.n_recv > 0) {
                k_halo_unpack<<<grid_of((long long)L.n_recv * b), 256, 0, d->stream>>>(
                    dst[p], d->jac[p]->ncp, L.d_recv, L.rbuf, L.n_recv, b);
                STS_LAUNCHED();
            }
    return STS_OK;
}

sts_status zero_ghosts(sts_dd_s *d, int p, double *x) {
    sts_jac_s *h = d->jac[p];
    const int c0 = d->plan[p]->n_owned;
    if (c0 >= h->ncp) return STS_OK;
    k_zero_cells<<<grid_of((long long)(h->ncp - c0) * h->b), 256, 0, d->stream>>>(x, h->ncp, c0, h->b);
    STS_LAUNCHED();
    return STS_OK;
}

// The library's kernels on the parts of this process.  Per part, the vectors
// are its handle's Krylov workspace; reductions sum the parts' totals on the
// host in part order, then over the processes.
struct GpuOps final : DdOps {
    sts_dd_s *d;
    int m, dir;
    GpuOps(sts_dd_s *d_, int m_, int dir_) : d(d_), m(m_), dir(dir_) {}
    double *vec(int p, int id) {
        Krylov &K = d->jac[p]->kry;
        const size_t n = (size_t)d->b * d->jac[p]->ncp;
        if (id <= m) return K.V + (size_t)id * n;
        if (id <= 2 * m) return K.Z + (size_t)(id - m - 1) * n;
        switch (id - 2 * m) {
            case 1: return K.w;
            case 2: return K.r;
            case 3: return K.xb;
            default: return K.bb;
        }
    }
    int np() const { return (int)d->jac.size(); }
    // the reduction output areas of part p's workspace: [0, m+2) dots, [m+2, 2m+4)
    // coefficients, [2m+4, ...) norms
    double *red(int p, int area) { return d->jac[p]->kry.red + (size_t)area * (m + 2); }
    double *pin(int p, int area) { return d->jac[p]->kry.h_pinned + (size_t)area * (m + 2); }
    sts_status gather_host(int area, int cnt, double *out) {
        for (int p = 0; p < np(); ++p)
            STS_CK(cudaMemcpyAsync(pin(p, area), red(p, area), sizeof(double) * cnt, cudaMemcpyDeviceToHost, d->stream));
        STS_CK(cudaStreamSynchronize(d->stream));
        for (int i = 0; i < cnt; ++i) out[i] = 0.0;
        for (int p = 0; p < np(); ++p)
            for (int i = 0; i < cnt; ++i) out[i] += pin(p, area)[i];
        return STS_OK;
    }
    sts_status to_device(int area, int cnt, const double *v) {
        STS_CK(cudaStreamSynchronize(d->stream));      // earlier copies out of the pinned area are done
        for (int p = 0; p < np(); ++p) {
            std::memcpy(pin(p, area), v, sizeof(double) * cnt);
            STS_CK(cudaMemcpyAsync(red(p, area), pin(p, area), sizeof(double) * cnt, cudaMemcpyHostToDevice,
                                   d->stream));
        }
        return STS_OK;
    }
    sts_status matvec(int in, int out) override {
        std::vector<const double *> src(np());
        std::vector<double *> dst(np());
        for (int p = 0; p < np(); ++p) {
            sts_jac_s *h = d->jac[p];
            src[p] = vec(p, in);
            dst[p] = h->vin;
            STS_CK(cudaMemcpyAsync(h->vin, src[p], sizeof(double) * d->b * h->ncp, cudaMemcpyDeviceToDevice,
                                   d->stream));
        }
        STS_TRY(halo(d, src, dst));
        for (int p = 0; p < np(); ++p) {
            STS_TRY(op_matvec64(d->jac[p], dir, d->jac[p]->vin, vec(p, out)));
            STS_TRY(zero_ghosts(d, p, vec(p, out)));
        }
        return STS_OK;
    }
    sts_status apply(int in, int out) override {
        for (int p = 0; p < np(); ++p) {
            STS_TRY(op_apply64(d->jac[p], dir, vec(p, in), vec(p, out)));
            STS_TRY(zero_ghosts(d, p, vec(p, out)));
        }
        return STS_OK;
    }
    sts_status copy(int out, int in) override {
        for (int p = 0; p < np(); ++p)
            STS_CK(cudaMemcpyAsync(vec(p, out), vec(p, in), sizeof(double) * d->b * d->jac[p]->ncp,
                                   cudaMemcpyDeviceToDevice, d->stream));
        return STS_OK;
    }
    sts_status sub(int out, int a, int b) override {
        for (int p = 0; p < np(); ++p) STS_TRY(kry_sub(d->jac[p], vec(p, out), vec(p, a), vec(p, b)));
        return STS_OK;
    }
    sts_status scale(int out, int in, double s) override {
        for (int p = 0; p < np(); ++p) {
            if (s == 0.0)
                STS_CK(cudaMemsetAsync(vec(p, out), 0, sizeof(double) * d->b * d->jac[p]->ncp, d->stream));
            else
                STS_TRY(kry_scale(d->jac[p], vec(p, out), vec(p, in), s));
        }
        return STS_OK;
    }
    sts_status dots(int v0, int k, int w, int self, double *out) override {
        for (int p = 0; p < np(); ++p) STS_TRY(kry_dots(d->jac[p], vec(p, v0), k, vec(p, w), self, red(p, 0)));
        return gather_host(0, k + (self ? 1 : 0), out);
    }
    sts_status update(int w, int v0, int k, const double *hc, int norm, double *out) override {
        STS_TRY(to_device(1, k, hc));
        for (int p = 0; p < np(); ++p)
            STS_TRY(kry_update(d->jac[p], vec(p, w), vec(p, v0), k, red(p, 1), norm, red(p, 2)));
        if (norm) return gather_host(2, 1, out);
        return STS_OK;
    }
    sts_status norm2(int v, double *out) override {
        for (int p = 0; p < np(); ++p) STS_TRY(kry_norm2(d->jac[p], vec(p, v), red(p, 2)));
        return gather_host(2, 1, out);
    }
    sts_status axpy(int x, int v0, int k, const double *y) override {
        if (k <= 0) return STS_OK;
        STS_TRY(to_device(1, k, y));
        for (int p = 0; p < np(); ++p) STS_TRY(kry_axpy(d->jac[p], vec(p, x), vec(p, v0), k, red(p, 1)));
        return STS_OK;
    }
    sts_status allreduce(double *vals, int n) override {
        if (!d->has_comm) return STS_OK;
        const int rc = d->comm.allreduce(d->comm.ctx, vals, n);
        return rc == 0 ? STS_OK : set_error(STS_ERR_COMM, "dd gmres: the allreduce callback returned %d", rc);
    }
};

sts_status dd_create_impl(const sts_dd_desc *desc, sts_dd_s **out) {
    if (!out) return set_error(STS_ERR_INVALID_ARG, "sts_dd_create: out is NULL");
    *out = nullptr;
    if (!desc || desc->n_parts < 1 || !desc->part_ids || !desc->jac || !desc->plans)
        return set_error(STS_ERR_INVALID_ARG, "sts_dd_create: bad descriptor");
    const int np = desc->n_parts;
    auto d = new sts_dd_s();
    d->has_comm = desc->comm != nullptr;
    if (d->has_comm) {
        d->comm = *desc->comm;
        if (!d->comm.exchange || !d->comm.allreduce) {
            delete d;
            return set_error(STS_ERR_INVALID_ARG, "sts_dd_create: comm needs both callbacks");
        }
    }
    std::map<int, int> local_of;
    for (int p = 0; p < np; ++p) {
        sts_jac_s *h = desc->jac[p];
        sts_dd_plan_s *P = desc->plans[p];
        const char *why = nullptr;
        if (!h || !P) why = "NULL handle or plan";
        else if (h->rep != STS_REP_FACTORED) why = "parts need the factored representation";
        else if (h->nc != (int)P->l2g.size()) why = "a handle's cell count differs from its plan's local cells";
        else if (P->part != desc->part_ids[p]) why = "part_ids differ from the plans' parts";
        else if (p > 0 && (h->stream != d->stream || h->b != d->b)) why = "parts need one stream and one block size";
        else if (local_of.count(P->part)) why = "a part is listed twice";
        if (why) {
            delete d;
            return set_error(STS_ERR_INVALID_ARG, "sts_dd_create: %s", why);
        }
        if (p == 0) {
            d->stream = h->stream;
            d->b = h->b;
        }
        local_of[P->part] = p;
        d->jac.push_back(h);
        d->plan.push_back(P);
        d->part_ids.push_back(P->part);
    }
    d->links.resize(np);
    sts_status st = STS_OK;
    auto upload_ints = [&](const int *a, int n, int **dptr) -> sts_status {
        STS_TRY(dd_alloc(d, reinterpret_cast<void **>(dptr), sizeof(int) * (size_t)std::max(n, 1)));
        if (n) STS_CK(cudaMemcpyAsync(*dptr, a, sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, d->stream));
        return STS_OK;
    };
    for (int p = 0; p < np && st == STS_OK; ++p) {
        sts_dd_plan_s *P = d->plan[p];
        for (size_t k = 0; k < P->nbr.size() && st == STS_OK; ++k) {
            sts_dd_s::Link L;
            L.peer = P->nbr[k];
            L.n_send = P->send_ptr[k + 1] - P->send_ptr[k];
            L.n_recv = P->recv_ptr[k + 1] - P->recv_ptr[k];
            auto it = local_of.find(L.peer);
            L.local_peer = it == local_of.end() ? -1 : it->second;
            if (L.local_peer < 0 && !d->has_comm) {
                st = set_error(STS_ERR_INVALID_ARG, "sts_dd_create: part %d neighbours part %d, which is not in this "
                               "process, and no comm was given", P->part, L.peer);
                break;
            }
            if ((st = upload_ints(P->send_cells.data() + P->send_ptr[k], L.n_send, &L.d_send)) != STS_OK) break;
            if ((st = upload_ints(P->recv_cells.data() + P->recv_ptr[k], L.n_recv, &L.d_recv)) != STS_OK) break;
            if (L.local_peer < 0) {
                if ((st = dd_alloc(d, reinterpret_cast<void **>(&L.sbuf), sizeof(double) * (size_t)L.n_send * d->b)) != STS_OK) break;
                if ((st = dd_alloc(d, reinterpret_cast<void **>(&L.rbuf), sizeof(double) * (size_t)L.n_recv * d->b)) != STS_OK) break;
            }
            d->links[p].push_back(L);
        }
    }
    // in-process neighbours: the peer's send list to this part is this part's receive list source
    for (int p = 0; p < np && st == STS_OK; ++p)
        for (auto &L : d->links[p]) {
            if (L.local_peer < 0) continue;
            const sts_dd_s::Link *back = nullptr;
            for (auto &M : d->links[L.local_peer])
                if (M.peer == d->part_ids[p]) back = &M;
            if (!back || back->n_send != L.n_recv) {
                st = set_error(STS_ERR_INVALID_ARG, "sts_dd_create: the plans of parts %d and %d disagree on their "
                               "halo (different partitions?)", d->part_ids[p], L.peer);
                break;
            }
            L.d_peer_send = back->d_send;
        }
    if (st == STS_OK) {
        cudaError_t e = cudaStreamSynchronize(d->stream);
        if (e != cudaSuccess) st = set_error(STS_ERR_CUDA, "sts_dd_create: %s", cudaGetErrorString(e));
    }
    if (st != STS_OK) {
        cudaStreamSynchronize(d->stream);
        dd_free(d);
        delete d;
        return st;
    }
    *out = d;
    return STS_OK;
}

sts_status dd_check_dir(sts_dd_s *d, int trans) {
    if (trans)
        for (auto h : d->jac)
            if (!h->has_T) return set_error(STS_ERR_INVALID_ARG, "dd: trans = 1 needs every part created with enable_transpose");
    return STS_OK;
}

sts_status dd_apply_impl(sts_dd_s *d, const double *const *x, double *const *y, int trans, bool matvec) {
    if (!x || !y) return set_error(STS_ERR_INVALID_ARG, "dd: NULL vector array");
    STS_TRY(dd_check_dir(d, trans));
    const int np = (int)d->jac.size(), dir = trans ? 1 : 0;
    for (int p = 0; p < np; ++p) {
        if (!x[p] || !y[p] || x[p] == y[p]) return set_error(STS_ERR_INVALID_ARG, "dd: NULL or overlapping vectors");
        if (!matvec && !d->jac[p]->smw.ready)
            return set_error(STS_ERR_NOT_SETUP, "dd: block-Jacobi used before sts_jac_bjacobi_setup on part %d",
                             d->part_ids[p]);
    }
    std::vector<const double *> src(np);
    std::vector<double *> dst(np);
    for (int p = 0; p < np; ++p) {
        STS_TRY(to_internal64(d->jac[p], x[p], d->jac[p]->vin));
        STS_TRY(zero_ghosts(d, p, d->jac[p]->vin));
        src[p] = d->jac[p]->vin;
        dst[p] = d->jac[p]->vin;
    }
    if (matvec) STS_TRY(halo(d, src, dst));
    for (int p = 0; p < np; ++p) {
        sts_jac_s *h = d->jac[p];
        if (matvec) STS_TRY(op_matvec64(h, dir, h->vin, h->vout));
        else STS_TRY(op_apply64(h, dir, h->vin, h->vout));
        STS_TRY(zero_ghosts(d, p, h->vout));
        STS_TRY(from_internal64(h, h->vout, y[p]));
    }
    return STS_OK;
}

sts_status dd_gmres_impl(sts_dd_s *d, const double *const *b, double *const *x, const sts_gmres_opts *o,
                         sts_gmres_info *info) {
    if (!b || !x) return set_error(STS_ERR_INVALID_ARG, "sts_dd_gmres_solve: NULL vector array");
    DdParams P;
    int dir = 0;
    STS_TRY(dd_options(o, true, &P, &dir));
    STS_TRY(dd_check_dir(d, dir));
    const int np = (int)d->jac.size();
    for (int p = 0; p < np; ++p) {
        if (!b[p] || !x[p] || b[p] == x[p]) return set_error(STS_ERR_INVALID_ARG, "sts_dd_gmres_solve: NULL or overlapping vectors");
        if (P.pre && !d->jac[p]->smw.ready)
            return set_error(STS_ERR_NOT_SETUP, "sts_dd_gmres_solve: block-Jacobi used before sts_jac_bjacobi_setup "
                             "on part %d", d->part_ids[p]);
        STS_TRY(kry_reserve(d->jac[p], P.m));
    }
    GpuOps ops(d, P.m, dir);
    for (int p = 0; p < np; ++p) {
        STS_TRY(to_internal64(d->jac[p], b[p], ops.vec(p, 2 * P.m + 4)));
        STS_TRY(zero_ghosts(d, p, ops.vec(p, 2 * P.m + 4)));
        STS_TRY(to_internal64(d->jac[p], x[p], ops.vec(p, 2 * P.m + 3)));
        STS_TRY(zero_ghosts(d, p, ops.vec(p, 2 * P.m + 3)));
    }
    const sts_status st = dd_gmres(ops, P, info);
    if (st == STS_OK || st == STS_ERR_NOT_CONVERGED) {
        for (int p = 0; p < np; ++p) {
            STS_TRY(zero_ghosts(d, p, ops.vec(p, 2 * P.m + 3)));
            STS_TRY(from_internal64(d->jac[p], ops.vec(p, 2 * P.m + 3), x[p]));
        }
        STS_CK(cudaStreamSynchronize(d->stream));
    }
    if (st == STS_OK || st == STS_ERR_NOT_CONVERGED || st == STS_ERR_NUMERIC)
        for (int p = 0; p < np; ++p) STS_TRY(check_device(d->jac[p]));
    return st;
}

}  // namespace
}  // namespace sts

using namespace sts;

#define STS_DD_GUARD(...)                                                         \
    try {                                                                         \
        __VA_ARGS__                                                               \
    } catch (const std::bad_alloc &) {                                            \
        return set_error(STS_ERR_ALLOC, "host allocation failed");                \
    } catch (...) {                                                               \
        return set_error(STS_ERR_INVALID_ARG, "unexpected exception");            \
    }

extern "C" {

sts_status sts_dd_plan_create(int n_cells, const int *block_indptr, const int *block_indices, int n_parts,
                              const int *part_of_cell, int part, sts_dd_plan_t *out) {
    if (!out) return set_error(STS_ERR_INVALID_ARG, "sts_dd_plan_create: out is NULL");
    *out = nullptr;
    STS_DD_GUARD(return plan_create(n_cells, block_indptr, block_indices, n_parts, part_of_cell, part, out);)
}

sts_status sts_dd_plan_sizes(sts_dd_plan_t P, sts_dd_sizes *z) {
    if (!P || !z) return set_error(STS_ERR_INVALID_ARG, "sts_dd_plan_sizes: NULL argument");
    z->n_owned = P->n_owned;
    z->n_local = (int)P->l2g.size();
    z->n_ghost = z->n_local - P->n_owned;
    z->nnzb = (int)P->bidx.size();
    z->n_neighbors = (int)P->nbr.size();
    z->n_send = (int)P->send_cells.size();
    z->n_recv = (int)P->recv_cells.size();
    return STS_OK;
}

sts_status sts_dd_plan_get(sts_dd_plan_t P, int *local_to_global, int *block_indptr, int *block_indices,
                           int *block_map, int *neighbors, int *send_ptr, int *send_cells, int *recv_ptr,
                           int *recv_cells) {
    if (!P) return set_error(STS_ERR_INVALID_ARG, "sts_dd_plan_get: plan is NULL");
    auto put = [](int *dst, const std::vector<int> &v) {
        if (dst && !v.empty()) std::memcpy(dst, v.data(), sizeof(int) * v.size());
    };
    put(local_to_global, P->l2g);
    put(block_indptr, P->bptr);
    put(block_indices, P->bidx);
    put(block_map, P->bmap);
    put(neighbors, P->nbr);
    put(send_ptr, P->send_ptr);
    put(send_cells, P->send_cells);
    put(recv_ptr, P->recv_ptr);
    put(recv_cells, P->recv_cells);
    return STS_OK;
}

sts_status sts_dd_plan_value_sizes(sts_dd_plan_t P, int nnz_d, int nnz_o, const int *pair_indptr, int r_diag,
                                   int r_off, long long *nnz_S, int *n_pairs, int *local_pair_indptr) {
    if (!P || nnz_d < 0 || nnz_o < 0 || r_diag < 0 || r_off < 0)
        return set_error(STS_ERR_INVALID_ARG, "sts_dd_plan_value_sizes: bad argument");
    STS_DD_GUARD({
        const std::vector<long long> pb = global_pair_base(P, pair_indptr, r_diag, r_off);
        const std::vector<long long> sb = global_s_base(P, nnz_d, nnz_o);
        long long s = 0, np_ = 0;
        if (local_pair_indptr) local_pair_indptr[0] = 0;
        for (size_t k = 0; k < P->bmap.size(); ++k) {
            const int g = P->bmap[k];
            s += sb[g + 1] - sb[g];
            np_ += pb[g + 1] - pb[g];
            if (local_pair_indptr) local_pair_indptr[k + 1] = (int)np_;
        }
        if (np_ > (1LL << 31) - 1) return set_error(STS_ERR_INVALID_ARG, "sts_dd_plan_value_sizes: too many pairs");
        if (nnz_S) *nnz_S = s;
        if (n_pairs) *n_pairs = (int)np_;
        return STS_OK;
    })
}

sts_status sts_dd_plan_gather(sts_dd_plan_t P, int block_size, int nnz_d, int nnz_o, const int *pair_indptr,
                              int r_diag, int r_off, const double *S, const double *U, const double *V,
                              double *S_local, double *U_local, double *V_local, int on_host, void *stream_) {
    NvtxRange nvtx_range("sts_dd_plan_gather");
    if (!P || block_size < 1 || !S || !S_local)
        return set_error(STS_ERR_INVALID_ARG, "sts_dd_plan_gather: bad argument");
    STS_DD_GUARD({
        const std::vector<long long> pb = global_pair_base(P, pair_indptr, r_diag, r_off);
        const std::vector<long long> sb = global_s_base(P, nnz_d, nnz_o);
        const int nb = (int)P->bmap.size();
        // segments: S, then U / V (the same segment list for both)
        std::vector<long long> ss(nb), sd(nb), ps, pd;
        std::vector<int> sl(nb), pl;
        long long so = 0, po = 0;
        for (int k = 0; k < nb; ++k) {
            const int g = P->bmap[k];
            ss[k] = sb[g];
            sd[k] = so;
            sl[k] = (int)(sb[g + 1] - sb[g]);
            so += sl[k];
            const long long cnt = (pb[g + 1] - pb[g]) * block_size;
            if (cnt > 0) {
                ps.push_back(pb[g] * block_size);
                pd.push_back(po);
                pl.push_back((int)cnt);
                po += cnt;
            }
        }
        if (po > 0 && (!U || !V || !U_local || !V_local))
            return set_error(STS_ERR_INVALID_ARG, "sts_dd_plan_gather: U or V is NULL");
        if (on_host) {
            for (int k = 0; k < nb; ++k) std::memcpy(S_local + sd[k], S + ss[k], sizeof(double) * sl[k]);
            for (size_t k = 0; k < pl.size(); ++k) {
                std::memcpy(U_local + pd[k], U + ps[k], sizeof(double) * pl[k]);
                std::memcpy(V_local + pd[k], V + ps[k], sizeof(double) * pl[k]);
            }
            return STS_OK;
        }
        cudaStream_t stream = static_cast<cudaStream_t>(stream_);
        const size_t nseg = std::max<size_t>(1, std::max((size_t)nb, pl.size()));
        long long *d_src = nullptr, *d_dst = nullptr;
        int *d_len = nullptr;
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&d_src), nseg * sizeof(long long), stream);
        if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&d_dst), nseg * sizeof(long long), stream);
        if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&d_len), nseg * sizeof(int), stream);
        auto run = [&](const std::vector<long long> &src_off, const std::vector<long long> &dst_off,
                       const std::vector<int> &len, const double *src, double *dst) -> cudaError_t {
            const int n = (int)len.size();
            if (n == 0) return cudaSuccess;
            cudaError_t r = cudaMemcpyAsync(d_src, src_off.data(), n * sizeof(long long), cudaMemcpyHostToDevice, stream);
            if (r == cudaSuccess) r = cudaMemcpyAsync(d_dst, dst_off.data(), n * sizeof(long long), cudaMemcpyHostToDevice, stream);
            if (r == cudaSuccess) r = cudaMemcpyAsync(d_len, len.data(), n * sizeof(int), cudaMemcpyHostToDevice, stream);
            if (r != cudaSuccess) return r;
            k_gather_segments<<<(int)std::min<long long>((n + 7) / 8, 152LL * 32), 256, 0, stream>>>(dst, src, d_src, d_dst,
                                                                                                   d_len, n);
            ::sts::g_launches.fetch_add(1, std::memory_order_relaxed);
            r = cudaGetLastError();
            // the host vectors must outlive the copies: wait before the next reuse
            if (r == cudaSuccess) r = cudaStreamSynchronize(stream);
            return r;
        };
        if (e == cudaSuccess) e = run(ss, sd, sl, S, S_local);
        if (e == cudaSuccess) e = run(ps, pd, pl, U, U_local);
        if (e == cudaSuccess) e = run(ps, pd, pl, V, V_local);
        if (d_src) cudaFreeAsync(d_src, stream);
        if (d_dst) cudaFreeAsync(d_dst, stream);
        if (d_len) cudaFreeAsync(d_len, stream);
        if (e != cudaSuccess) return set_error(STS_ERR_CUDA, "sts_dd_plan_gather: %s", cudaGetErrorString(e));
        return STS_OK;
    })
}

sts_status sts_dd_plan_destroy(sts_dd_plan_t P) {
    delete P;
    return STS_OK;
}

sts_status sts_dd_create(const sts_dd_desc *desc, sts_dd_t *out) {
    NvtxRange nvtx_range("sts_dd_create");
    STS_DD_GUARD(return dd_create_impl(desc, out);)
}

sts_status sts_dd_matvec(sts_dd_t d, const double *const *x, double *const *y, int trans) {
    NvtxRange nvtx_range("sts_dd_matvec");
    if (!d) return set_error(STS_ERR_INVALID_ARG, "sts_dd_matvec: handle is NULL");
    STS_DD_GUARD(return dd_apply_impl(d, x, y, trans, true);)
}

sts_status sts_dd_bjacobi_apply(sts_dd_t d, const double *const *x, double *const *z, int trans) {
    NvtxRange nvtx_range("sts_dd_bjacobi_apply");
    if (!d) return set_error(STS_ERR_INVALID_ARG, "sts_dd_bjacobi_apply: handle is NULL");
    STS_DD_GUARD(return dd_apply_impl(d, x, z, trans, false);)
}

sts_status sts_dd_gmres_solve(sts_dd_t d, const double *const *b, double *const *x, const sts_gmres_opts *opts,
                              sts_gmres_info *info) {
    NvtxRange nvtx_range("sts_dd_gmres_solve");
    if (!d) return set_error(STS_ERR_INVALID_ARG, "sts_dd_gmres_solve: handle is NULL");
    STS_DD_GUARD(return dd_gmres_impl(d, b, x, opts, info);)
}

sts_status sts_dd_destroy(sts_dd_t d) {
    if (!d) return STS_OK;
    cudaStreamSynchronize(d->stream);
    dd_free(d);
    delete d;
    return STS_OK;
}

sts_status sts_dd_gmres_ops(const sts_dd_ops *ops, const sts_gmres_opts *opts, sts_gmres_info *info) {
    NvtxRange nvtx_range("sts_dd_gmres_ops");
    if (!ops || !ops->matvec || !ops->apply || !ops->copy || !ops->sub || !ops->scale || !ops->dots ||
        !ops->update || !ops->norm2 || !ops->axpy || !ops->allreduce)
        return set_error(STS_ERR_INVALID_ARG, "sts_dd_gmres_ops: every callback is needed");
    STS_DD_GUARD({
        DdParams P;
        int dir = 0;
        STS_TRY(dd_options(opts, false, &P, &dir));
        CbOps cb(ops);
        return dd_gmres(cb, P, info);
    })
}

}  // extern "C"
