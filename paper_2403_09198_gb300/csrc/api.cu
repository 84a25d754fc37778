// api.cu -- the C ABI of libsts (declared in include/sts.h): validation of the
// problem statement, host-side construction of the kernels' plans, device
// memory ownership and the entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "ring.cuh"
#include "sts_internal.h"

namespace sts {

static thread_local char g_err[1024] = "";
std::atomic<unsigned long long> g_launches{0};

sts_status set_error(sts_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

sts_status dev_alloc(sts_jac_s *h, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_error(STS_ERR_ALLOC, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    h->allocs.push_back(DevBuf{*p, bytes});
    h->bytes += bytes;
    return STS_OK;
}

void dev_free(sts_jac_s *h, void *p) {
    if (!p) return;
    for (size_t i = 0; i < h->allocs.size(); ++i)
        if (h->allocs[i].p == p) {
            cudaFree(p);
            h->bytes -= h->allocs[i].bytes;
            h->allocs.erase(h->allocs.begin() + (long)i);
            return;
        }
}

// Band half-width w if rows p < N = b - kStructNF hold exactly the level band
// |p - q| <= w followed by the kStructNF flow columns and the last kStructNF
// rows are dense; -1 if the pattern is not of that family.
int struct_band(int b, const std::vector<int> &ptr, const std::vector<int> &idx) {
    const int N = b - kStructNF;
    if (N < 1) return -1;
    for (int r = N; r < b; ++r) {
        if (ptr[r + 1] - ptr[r] != b) return -1;
        for (int e = ptr[r]; e < ptr[r + 1]; ++e)
            if (idx[e] != e - ptr[r]) return -1;
    }
    for (int w = 0; w <= kStructMaxW; ++w) {
        bool ok = true;
        for (int p = 0; p < N && ok; ++p) {
            const int lo = std::max(0, p - w), hi = std::min(N - 1, p + w);
            if (ptr[p + 1] - ptr[p] != (hi - lo + 1) + kStructNF) {
                ok = false;
                break;
            }
            int e = ptr[p];
            for (int q = lo; q <= hi; ++q, ++e) ok = ok && idx[e] == q;
            for (int f = 0; f < kStructNF; ++f, ++e) ok = ok && idx[e] == N + f;
        }
        if (ok) return w;
    }
    return -1;
}

namespace {

sts_status check_csr(const int *ptr, const int *idx, int rows, int cols, bool need_diag, const char *what) {
    if (!ptr) return set_error(STS_ERR_INVALID_ARG, "%s: indptr is NULL", what);
    if (ptr[0] != 0) return set_error(STS_ERR_INVALID_ARG, "%s: indptr[0] must be 0", what);
    for (int i = 0; i < rows; ++i)
        if (ptr[i + 1] < ptr[i]) return set_error(STS_ERR_INVALID_ARG, "%s: indptr decreases at row %d", what, i);
    if (ptr[rows] > 0 && !idx) return set_error(STS_ERR_INVALID_ARG, "%s: indices is NULL", what);
    for (int i = 0; i < rows; ++i) {
        bool diag = false;
        for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
            const int j = idx[e];
            if (j < 0 || j >= cols)
                return set_error(STS_ERR_INVALID_ARG, "%s: column %d out of range in row %d", what, j, i);
            if (e > ptr[i] && j <= idx[e - 1])
                return set_error(STS_ERR_INVALID_ARG, "%s: row %d not strictly ascending", what, i);
            diag = diag || j == i;
        }
        if (need_diag && !diag) return set_error(STS_ERR_INVALID_ARG, "%s: row %d has no diagonal entry", what, i);
    }
    return STS_OK;
}

// Transpose of a b x b CSR pattern; src[e'] = entry index of the original entry.
void transpose_pattern(int b, const std::vector<int> &ptr, const std::vector<int> &idx, std::vector<int> &tptr,
                       std::vector<int> &tidx, std::vector<int> &src) {
    const int nnz = ptr[b];
    tptr.assign(b + 1, 0);
    for (int e = 0; e < nnz; ++e) tptr[idx[e] + 1]++;
    for (int q = 0; q < b; ++q) tptr[q + 1] += tptr[q];
    tidx.assign(nnz, 0);
    src.assign(nnz, 0);
    std::vector<int> fill(tptr.begin(), tptr.end() - 1);
    for (int p = 0; p < b; ++p)
        for (int e = ptr[p]; e < ptr[p + 1]; ++e) {
            const int t = fill[idx[e]]++;
            tidx[t] = p;
            src[t] = e;
        }
}

// Build the plan of one matvec direction (dir 0: y = J x, dir 1: y = J^T x).
sts_status build_plan(sts_jac_s *h, int dir, bool with_streams) {
    MvPlan &P = h->mv[dir];
    const int nc = h->nc, b = h->b, nt = h->n_tiles;
    // block slots of every cell
    std::vector<int> cptr(nc + 1, 0), cblk, cnbr;
    if (dir == 0) {
        for (int c = 0; c < nc; ++c) {
            int kd = -1;
            for (int k = h->bptr[c]; k < h->bptr[c + 1]; ++k)
                if (h->bidx[k] == c) kd = k;
            cblk.push_back(kd);
            cnbr.push_back(c);
            for (int k = h->bptr[c]; k < h->bptr[c + 1]; ++k)
                if (h->bidx[k] != c) {
                    cblk.push_back(k);
                    cnbr.push_back(h->bidx[k]);
                }
            cptr[c + 1] = (int)cblk.size();
        }
    } else {
        std::vector<std::vector<std::pair<int, int>>> col(nc);
        for (int i = 0; i < nc; ++i)
            for (int k = h->bptr[i]; k < h->bptr[i + 1]; ++k) col[h->bidx[k]].push_back({i, k});
        for (int c = 0; c < nc; ++c) {
            int kd = -1;
            for (auto &ik : col[c])
                if (ik.first == c) kd = ik.second;
            cblk.push_back(kd);
            cnbr.push_back(c);
            for (auto &ik : col[c])
                if (ik.first != c) {
                    cblk.push_back(ik.second);
                    cnbr.push_back(ik.first);
                }
            cptr[c + 1] = (int)cblk.size();
        }
    }
    int n_slots = 1;
    for (int c = 0; c < nc; ++c) n_slots = std::max(n_slots, cptr[c + 1] - cptr[c]);
    if (n_slots > kMaxSlots)
        return set_error(STS_ERR_INVALID_ARG, "a block %s holds %d blocks; at most %d are supported",
                         dir == 0 ? "row" : "column", n_slots, kMaxSlots);
    P.n_slots = n_slots;
    std::vector<int> nbr((size_t)nt * n_slots * kTile, -1), blk((size_t)nt * n_slots * kTile, -1);
    std::vector<unsigned> mask(nt, 0u);
    for (int c = 0; c < nc; ++c) {
        const int t = c / kTile, lane = c % kTile;
        for (int s = 0; s < cptr[c + 1] - cptr[c]; ++s) {
            nbr[((size_t)t * n_slots + s) * kTile + lane] = cnbr[cptr[c] + s];
            blk[((size_t)t * n_slots + s) * kTile + lane] = cblk[cptr[c] + s];
            mask[t] |= 1u << s;
        }
    }
    // patterns of this direction
    std::vector<int> kp[2], ki[2], ks[2];
    if (dir == 0) {
        kp[0] = h->dptr; ki[0] = h->didx; kp[1] = h->optr; ki[1] = h->oidx;
        ks[0].resize(h->nnz_d); ks[1].resize(h->nnz_o);
        for (int e = 0; e < h->nnz_d; ++e) ks[0][e] = e;
        for (int e = 0; e < h->nnz_o; ++e) ks[1][e] = e;
    } else {
        transpose_pattern(b, h->dptr, h->didx, kp[0], ki[0], ks[0]);
        transpose_pattern(b, h->optr, h->oidx, kp[1], ki[1], ks[1]);
    }
    // pair slots
    std::vector<int> pslot_slot, pslot_local;
    for (int s = 0; s < n_slots; ++s) {
        const int r = s == 0 ? h->r_diag : h->r_off;
        for (int l = 0; l < r; ++l) {
            pslot_slot.push_back(s);
            pslot_local.push_back(l);
        }
    }
    P.n_pslots = (int)pslot_slot.size();
    // structured family?  (diagonal kind: band wd; neighbour kind: band 0)
    const int wd = struct_band(b, kp[0], ki[0]);
    const int wo = n_slots > 1 ? struct_band(b, kp[1], ki[1]) : 0;
    P.structured = wd >= 0 && wo == 0 && n_slots <= kStructMaxSlots;
    std::vector<long long> row_off(b + 1, 0);
    std::vector<int> pos_kind, pos_arg;
    std::vector<int> grp(1, 0);
    std::vector<int> dtask_slot, dpos_kind, dpos_arg;
    const int Lp = (b + 15) / 16 * 16;      // dot length padded to the largest register chunk
    P.Lp = Lp;
    if (P.structured) {
        const int NF = kStructNF, N = b - NF;
        std::vector<int> ent[2];
        for (int k = 0; k < 2; ++k) {
            ent[k].assign((size_t)b * b, -1);
            for (int p = 0; p < b; ++p)
                for (int e = kp[k][p]; e < kp[k][p + 1]; ++e) ent[k][(size_t)p * b + ki[k][e]] = e;
        }
        auto push = [&](int kind, int arg) {
            pos_kind.push_back(kind);
            pos_arg.push_back(arg);
        };
        for (int p = 0; p < N; ++p) {
            for (int k = 0; k <= 2 * wd; ++k) {
                const int q = p - wd + k;
                if (q >= 0 && q < N) push(0, ent[0][(size_t)p * b + q]);
                else push(kPosZero, 0);
            }
            for (int f = 0; f < NF; ++f) push(0, ent[0][(size_t)p * b + N + f]);
            for (int sl = 1; sl < n_slots; ++sl) {
                push(sl, h->nnz_d + ent[1][(size_t)p * b + p]);
                for (int f = 0; f < NF; ++f) push(sl, h->nnz_d + ent[1][(size_t)p * b + N + f]);
            }
            for (int k = 0; k < P.n_pslots; ++k) push(-1 - k, p);
        }
        for (int f = 0; f < NF; ++f)
            for (int k = 0; k < P.n_pslots; ++k) push(-1 - k, N + f);
        // pass-1 tasks: pair dots, then the dense flow rows of every slot
        for (int k = 0; k < P.n_pslots; ++k) {
            dtask_slot.push_back(pslot_slot[k]);
            for (int q = 0; q < Lp; ++q) {
                dpos_kind.push_back(q < b ? -1 - k : kPosZero);
                dpos_arg.push_back(q < b ? q : 0);
            }
        }
        for (int f = 0; f < NF; ++f)
            for (int sl = 0; sl < n_slots; ++sl) {
                const int kd = sl == 0 ? 0 : 1;
                dtask_slot.push_back(sl);
                for (int q = 0; q < Lp; ++q) {
                    dpos_kind.push_back(q < b ? sl : kPosZero);
                    dpos_arg.push_back(q < b ? (kd ? h->nnz_d : 0) + ent[kd][(size_t)(N + f) * b + q] : 0);
                }
            }
        P.s_wd = wd;
        P.sN = N;
        P.s_rl = (2 * wd + 1 + NF) + (n_slots - 1) * (1 + NF) + P.n_pslots;
        P.s_gl = std::max(1, (180 + P.s_rl / 2) / P.s_rl);    // about 180 FMAs per lane and warp item
        P.n_lgroups = (N + P.s_gl - 1) / P.s_gl;
        P.n_groups = P.n_lgroups + 1;
        P.tile_len = (long long)pos_kind.size();
        if (P.tile_len != (long long)N * P.s_rl + (long long)NF * P.n_pslots)
            return set_error(STS_ERR_INVALID_ARG, "internal: structured stream size");
        for (int g = 1; g <= P.n_lgroups; ++g) grp.push_back(std::min(N, g * P.s_gl));
        grp.push_back(b);
    } else {
        // main stream order and row offsets
        long long maxlen = 0;
        for (int p = 0; p < b; ++p) {
            const long long start = (long long)pos_kind.size();
            for (int s = 0; s < n_slots; ++s) {
                const int kind = s == 0 ? 0 : 1;
                const int off = kind ? h->nnz_d : 0;
                for (int e = kp[kind][p]; e < kp[kind][p + 1]; ++e) {
                    pos_kind.push_back(s);
                    pos_arg.push_back(off + e);
                }
            }
            for (int k = 0; k < P.n_pslots; ++k) {
                pos_kind.push_back(-1 - k);
                pos_arg.push_back(p);
            }
            row_off[p + 1] = (long long)pos_kind.size();
            maxlen = std::max(maxlen, row_off[p + 1] - start);
        }
        P.tile_len = row_off[b];
        // row groups: contiguous rows, balanced by stream length
        const long long target = std::max(maxlen, (P.tile_len + 15) / 16);
        long long cur = 0;
        for (int p = 0; p < b; ++p) {
            const long long len = row_off[p + 1] - row_off[p];
            if (cur > 0 && cur + len > target) {
                grp.push_back(p);
                cur = 0;
            }
            cur += len;
        }
        grp.push_back(b);
        P.n_groups = (int)grp.size() - 1;
        for (int k = 0; k < P.n_pslots; ++k) {
            dtask_slot.push_back(pslot_slot[k]);
            for (int q = 0; q < Lp; ++q) {
                dpos_kind.push_back(q < b ? -1 - k : kPosZero);
                dpos_arg.push_back(q < b ? q : 0);
            }
        }
    }
    P.n_dtasks = (int)dtask_slot.size();
    P.h_grp_rows = grp;
    P.h_row_off = row_off;
    P.h_pslot_slot = pslot_slot;
    P.h_blk = blk;
    std::vector<int> pat_ptr(2 * (b + 1)), pat_idx, pat_src;
    for (int k = 0; k < 2; ++k) {
        std::copy(kp[k].begin(), kp[k].end(), pat_ptr.begin() + k * (b + 1));
        pat_idx.insert(pat_idx.end(), ki[k].begin(), ki[k].end());
        pat_src.insert(pat_src.end(), ks[k].begin(), ks[k].end());
    }
    STS_TRY(upload(h, &P.nbr, nbr));
    STS_TRY(upload(h, &P.blk, blk));
    STS_TRY(upload(h, &P.slot_mask, mask));
    STS_TRY(upload(h, &P.grp_rows, grp));
    STS_TRY(upload(h, &P.row_off, row_off));
    STS_TRY(upload(h, &P.pslot_slot, pslot_slot));
    STS_TRY(upload(h, &P.pslot_local, pslot_local));
    STS_TRY(upload(h, &P.dtask_slot, dtask_slot));
    STS_TRY(upload(h, &P.pat_ptr, pat_ptr));
    STS_TRY(upload(h, &P.pat_idx, pat_idx));
    STS_TRY(upload(h, &P.pat_src, pat_src));
    if (with_streams) {
        if (b > 0xffff) return set_error(STS_ERR_INVALID_ARG, "block_size above 65535 is not supported");
        std::vector<unsigned> desc(P.structured ? 1 : pos_kind.size(), 0u);
        if (!P.structured) {
            for (int p = 0; p < b; ++p)
                for (long long q = row_off[p]; q < row_off[p + 1]; ++q) {
                    const int kind = pos_kind[q];
                    unsigned d;
                    if (kind >= 0) {
                        const int kd = kind == 0 ? 0 : 1;
                        const int e = pos_arg[q] - (kd ? h->nnz_d : 0);
                        d = (unsigned)ki[kd][e] | ((unsigned)kind << 16);
                    } else {
                        d = (unsigned)(-1 - kind) | kDescPair;
                    }
                    if (q == row_off[p + 1] - 1) d |= kDescEnd;
                    desc[q] = d;
                }
            // a row with no stream positions would never be written
            for (int p = 0; p < b; ++p)
                if (row_off[p + 1] == row_off[p])
                    return set_error(STS_ERR_INVALID_ARG, "row %d of the Jacobian blocks is empty in every slot; "
                                     "add an explicit zero to the pattern", p);
        }
        STS_TRY(upload(h, &P.desc, desc));
        STS_TRY(upload(h, &P.pos_kind, pos_kind));
        STS_TRY(upload(h, &P.pos_arg, pos_arg));
        STS_TRY(upload(h, &P.dpos_kind, dpos_kind));
        STS_TRY(upload(h, &P.dpos_arg, dpos_arg));
        const size_t nm = (size_t)nt * P.tile_len * kTile;
        const size_t nd = (size_t)nt * P.n_dtasks * Lp * kTile;
        STS_TRY(dalloc(h, &P.main64, nm));
        STS_TRY(dalloc(h, &P.dotv64, nd));
        if (h->dtype == STS_MIXED) {
            STS_TRY(dalloc(h, &P.main32, nm));
            STS_TRY(dalloc(h, &P.dotv32, nd));
        }
    }
    return STS_OK;
}

// Adjoint bookkeeping: owner cells of every block and pair, and where each
// pair's dot lands in the pass-1 output of either direction.
sts_status build_grad_tables(sts_jac_s *h) {
    std::vector<int> brow(h->nnzb), bcol(h->nnzb);
    for (int i = 0; i < h->nc; ++i)
        for (int k = h->bptr[i]; k < h->bptr[i + 1]; ++k) {
            brow[k] = i;
            bcol[k] = h->bidx[k];
        }
    std::vector<int> erow(h->nnz_d + h->nnz_o);
    for (int p = 0; p < h->b; ++p) {
        for (int e = h->dptr[p]; e < h->dptr[p + 1]; ++e) erow[e] = p;
        for (int e = h->optr[p]; e < h->optr[p + 1]; ++e) erow[h->nnz_d + e] = p;
    }
    std::vector<int> prow(h->n_pairs), pcol(h->n_pairs), pcN(h->n_pairs, 0), pcT(h->n_pairs, 0);
    for (int k = 0; k < h->nnzb; ++k)
        for (int pr = h->pbase[k]; pr < h->pbase[k + 1]; ++pr) {
            prow[pr] = brow[k];
            pcol[pr] = bcol[k];
        }
    for (int dir = 0; dir < 2; ++dir) {
        const MvPlan &P = h->mv[dir];
        const std::vector<int> &hblk = P.h_blk;
        std::vector<int> &dst = dir == 0 ? pcN : pcT;
        for (int t = 0; t < h->n_tiles; ++t)
            for (int ps = 0; ps < P.n_pslots; ++ps) {
                const int s = P.h_pslot_slot[ps];
                int local = 0;
                for (int q = 0; q < ps; ++q)
                    if (P.h_pslot_slot[q] == s) ++local;
                for (int lane = 0; lane < kTile; ++lane) {
                    const int k = hblk[((size_t)t * P.n_slots + s) * kTile + lane];
                    if (k < 0 || local >= h->pbase[k + 1] - h->pbase[k]) continue;   // padding pair
                    dst[h->pbase[k] + local] = (int)(((size_t)t * P.n_dtasks + ps) * kTile + lane);
                }
            }
    }
    STS_TRY(upload(h, &h->g_blk_row, brow));
    STS_TRY(upload(h, &h->g_blk_col, bcol));
    STS_TRY(upload(h, &h->g_erow, erow));
    STS_TRY(upload(h, &h->g_pair_row, prow));
    STS_TRY(upload(h, &h->g_pair_col, pcol));
    STS_TRY(upload(h, &h->g_pair_cN, pcN));
    STS_TRY(upload(h, &h->g_pair_cT, pcT));
    return STS_OK;
}

sts_status load_values(sts_jac_s *h, const double *S, const double *U, const double *V, int on_host) {
    const double *dS = S, *dU = U, *dV = V;
    const size_t nS = (size_t)h->nnz_S, nP = (size_t)h->n_pairs * h->b;
    if (on_host) {
        // one staging buffer per handle, allocated on the first update from host
        // memory and kept: a fresh allocation per update would map and unmap the
        // whole value array every time
        if (!h->staging) STS_TRY(dalloc(h, &h->staging, nS + 2 * nP + 1));
        double *tmp = h->staging;
        STS_CK(cudaMemcpyAsync(tmp, S, nS * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        if (nP) {
            STS_CK(cudaMemcpyAsync(tmp + nS, U, nP * sizeof(double), cudaMemcpyHostToDevice, h->stream));
            STS_CK(cudaMemcpyAsync(tmp + nS + nP, V, nP * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        }
        dS = tmp;
        dU = tmp + nS;
        dV = tmp + nS + nP;
    }
    sts_status st = STS_OK;
    if (h->rep == STS_REP_FACTORED) {
        st = mv_repack(h, 0, dS, dU, dV);
        if (st == STS_OK && h->has_T) st = mv_repack(h, 1, dS, dU, dV);
        if (st == STS_OK) st = smw_repack(h, dS, dU, dV);
        h->streams_dirty = true;
    } else {
        st = dense_build(h, dS, dU, dV);
    }
    return st;
}

void free_all(sts_jac_s *h) {
    for (auto &b : h->allocs) cudaFree(b.p);
    h->allocs.clear();
    if (h->kry.h_pinned) cudaFreeHost(h->kry.h_pinned);
    h->kry.h_pinned = nullptr;
    if (h->kry.g_pinned) cudaFreeHost(h->kry.g_pinned);
    h->kry.g_pinned = nullptr;
    for (auto &row : h->kry.gexec)
        for (auto &ge : row) {
            if (ge) cudaGraphExecDestroy(ge);
            ge = nullptr;
        }
}

bool layout_ok(int l) { return l == STS_LAYOUT_CELL_MAJOR || l == STS_LAYOUT_COMPONENT_MAJOR; }

sts_status create_impl(const sts_jac_desc *d, sts_jac_t *out) {
    if (!out) return set_error(STS_ERR_INVALID_ARG, "sts_jac_create: out is NULL");
    *out = nullptr;
    if (!d) return set_error(STS_ERR_INVALID_ARG, "sts_jac_create: desc is NULL");
    if (d->n_cells < 1 || d->block_size < 1)
        return set_error(STS_ERR_INVALID_ARG, "sts_jac_create: n_cells and block_size must be >= 1");
    if (d->dtype != STS_F64 && d->dtype != STS_MIXED)
        return set_error(STS_ERR_INVALID_ARG, "sts_jac_create: dtype must be STS_F64 or STS_MIXED");
    if (!layout_ok(d->vec_layout)) return set_error(STS_ERR_INVALID_ARG, "sts_jac_create: unknown vec_layout");
    if (d->representation != STS_REP_FACTORED && d->representation != STS_REP_DENSE_BSR)
        return set_error(STS_ERR_INVALID_ARG, "sts_jac_create: unknown representation");
    if (d->r_diag < 0 || d->r_off < 0) return set_error(STS_ERR_INVALID_ARG, "sts_jac_create: negative pair count");
    if (d->representation == STS_REP_DENSE_BSR && (d->dtype != STS_F64 || d->enable_transpose))
        return set_error(STS_ERR_INVALID_ARG, "sts_jac_create: the dense-BSR baseline is FP64, forward only");
    const int nc = d->n_cells, b = d->block_size;
    if ((long long)nc * b > (1LL << 31) - 1)
        return set_error(STS_ERR_INVALID_ARG, "sts_jac_create: n_cells * block_size must fit in int32");
    STS_TRY(check_csr(d->block_indptr, d->block_indices, nc, nc, true, "block structure"));
    STS_TRY(check_csr(d->d_indptr, d->d_indices, b, b, true, "diagonal-block pattern"));
    STS_TRY(check_csr(d->o_indptr, d->o_indices, b, b, false, "off-diagonal-block pattern"));
    const int nnzb = d->block_indptr[nc];
    // Pairs per block: uniform per block kind, or the caller's pair_indptr.  The
    // handle stores every block with the largest count of its kind.
    int r_diag = d->r_diag, r_off = d->r_off;
    long long n_pairs = (long long)nc * r_diag + (long long)(nnzb - nc) * r_off;
    if (d->pair_indptr) {
        const int *pp = d->pair_indptr;
        if (pp[0] != 0) return set_error(STS_ERR_INVALID_ARG, "sts_jac_create: pair_indptr[0] must be 0");
        r_diag = r_off = 0;
        for (int i = 0; i < nc; ++i)
            for (int k = d->block_indptr[i]; k < d->block_indptr[i + 1]; ++k) {
                const int cnt = pp[k + 1] - pp[k];
                if (cnt < 0)
                    return set_error(STS_ERR_INVALID_ARG, "sts_jac_create: pair_indptr decreases at block %d", k);
                int &rmax = d->block_indices[k] == i ? r_diag : r_off;
                rmax = std::max(rmax, cnt);
            }
        n_pairs = pp[nnzb];
    }
    if (n_pairs > (1LL << 31) - 1) return set_error(STS_ERR_INVALID_ARG, "sts_jac_create: too many pairs");
    if (!d->S) return set_error(STS_ERR_INVALID_ARG, "sts_jac_create: S is NULL");
    if (n_pairs > 0 && (!d->U || !d->V)) return set_error(STS_ERR_INVALID_ARG, "sts_jac_create: U or V is NULL");

    sts_jac_s *h = new sts_jac_s();
    h->nc = nc;
    h->b = b;
    h->N = d->n_levels;
    h->dtype = d->dtype;
    h->layout = d->vec_layout;
    h->rep = d->representation;
    h->r_diag = r_diag;
    h->r_off = r_off;
    h->nnz_d = d->d_indptr[b];
    h->nnz_o = d->o_indptr[b];
    h->nnzb = nnzb;
    h->n_pairs = (int)n_pairs;
    h->n_tiles = (nc + kTile - 1) / kTile;
    h->ncp = h->n_tiles * kTile;
    h->has_T = d->enable_transpose != 0;
    h->stream = static_cast<cudaStream_t>(d->stream);
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || h->nsm < 1 ||
            cudaDeviceGetAttribute(&h->l2_bytes, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
            delete h;
            return set_error(STS_ERR_CUDA, "sts_jac_create: cannot query the device");
        }
        h->device = dev;
    }
    h->bptr.assign(d->block_indptr, d->block_indptr + nc + 1);
    h->bidx.assign(d->block_indices, d->block_indices + nnzb);
    h->dptr.assign(d->d_indptr, d->d_indptr + b + 1);
    h->didx.assign(d->d_indices, d->d_indices + h->nnz_d);
    h->optr.assign(d->o_indptr, d->o_indptr + b + 1);
    if (h->nnz_o) h->oidx.assign(d->o_indices, d->o_indices + h->nnz_o);
    h->soff.assign(nnzb + 1, 0);
    h->pbase.assign(nnzb + 1, 0);
    for (int i = 0; i < nc; ++i)
        for (int k = h->bptr[i]; k < h->bptr[i + 1]; ++k) {
            const bool diag = h->bidx[k] == i;
            h->soff[k + 1] = h->soff[k] + (diag ? h->nnz_d : h->nnz_o);
            h->pbase[k + 1] = d->pair_indptr ? d->pair_indptr[k + 1]
                                             : h->pbase[k] + (diag ? h->r_diag : h->r_off);
        }
    h->nnz_S = h->soff[nnzb];
    sts_status st = STS_OK;
    do {
        if ((st = upload(h, &h->d_soff, h->soff)) != STS_OK) break;
        if ((st = upload(h, &h->d_pbase, h->pbase)) != STS_OK) break;
        const bool fact = h->rep == STS_REP_FACTORED;
        if ((st = build_plan(h, 0, fact)) != STS_OK) break;
        if (h->has_T && (st = build_plan(h, 1, true)) != STS_OK) break;
        const size_t n = (size_t)b * h->ncp;
        if ((st = dalloc(h, &h->vin, n)) != STS_OK) break;
        if ((st = dalloc(h, &h->vout, n)) != STS_OK) break;
        if ((st = dalloc(h, &h->d_err, 1)) != STS_OK) break;
        if ((st = dalloc(h, &h->d_sched, 2)) != STS_OK) break;
        if (cudaMemsetAsync(h->d_sched, 0, 2 * sizeof(unsigned), h->stream) != cudaSuccess ||
            cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream) != cudaSuccess) {
            st = set_error(STS_ERR_CUDA, "sts_jac_create: cudaMemsetAsync failed");
            break;
        }
        const int nps = std::max(h->mv[0].n_dtasks, h->mv[1].n_dtasks);
        if ((st = dalloc(h, &h->c64, (size_t)h->n_tiles * nps * kTile + 1)) != STS_OK) break;
        if (h->dtype == STS_MIXED) {
            if ((st = dalloc(h, &h->vin32, n)) != STS_OK) break;
            if ((st = dalloc(h, &h->vout32, n)) != STS_OK) break;
            if ((st = dalloc(h, &h->c32, (size_t)h->n_tiles * nps * kTile + 1)) != STS_OK) break;
        }
        if (fact && (st = smw_build(h)) != STS_OK) break;
        if (fact && h->has_T && (st = build_grad_tables(h)) != STS_OK) break;
        if ((st = load_values(h, d->S, d->U, d->V, d->values_on_host)) != STS_OK) break;
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) {
            st = set_error(STS_ERR_CUDA, "sts_jac_create: %s", cudaGetErrorString(e));
            break;
        }
    } while (false);
    if (st != STS_OK) {
        cudaStreamSynchronize(h->stream);
        free_all(h);
        delete h;
        return st;
    }
    *out = h;
    return STS_OK;
}

// Run an operator on public-layout vectors through the internal layout.  With
// the component-major layout and no padding cells the kernels work in place.
template <typename T, typename F>
sts_status with_layout(sts_jac_s *h, const T *x, T *y, T *bin, T *bout, F op) {
    if (h->layout == STS_LAYOUT_COMPONENT_MAJOR && h->nc == h->ncp) return op(x, y);
    if constexpr (sizeof(T) == 8) {
        STS_TRY(to_internal64(h, reinterpret_cast<const double *>(x), reinterpret_cast<double *>(bin)));
        STS_TRY(op(bin, bout));
        return from_internal64(h, reinterpret_cast<const double *>(bout), reinterpret_cast<double *>(y));
    } else {
        STS_TRY(to_internal32(h, reinterpret_cast<const float *>(x), reinterpret_cast<float *>(bin)));
        STS_TRY(op(bin, bout));
        return from_internal32(h, reinterpret_cast<const float *>(bout), reinterpret_cast<float *>(y));
    }
}

sts_status check_handle(sts_jac_t h, const void *a, const void *b, const char *fn) {
    if (!h) return set_error(STS_ERR_INVALID_ARG, "%s: handle is NULL", fn);
    if (!a || !b) return set_error(STS_ERR_INVALID_ARG, "%s: NULL vector", fn);
    if (a == b) return set_error(STS_ERR_INVALID_ARG, "%s: input and output must not overlap", fn);
    return STS_OK;
}

// One warp waits, through the rings' bounded wait, on a phase nothing completes.
__global__ void k_wait_selftest(int *flag) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_addr(&bar), 1);
        mbar_init_fence();
    }
    __syncwarp();
    const bool done = mbar_wait_bounded(smem_addr(&bar), 0u);
    if (threadIdx.x == 0) *flag = done ? 2 : 1;
}

}  // namespace

// A bounded device wait (bulk copies into shared memory) gave up since the
// last check: report it once and clear the flag.
sts_status check_device(sts_jac_s *h) {
    if (!h->d_err) return STS_OK;
    int flag = 0;
    STS_CK(cudaMemcpyAsync(&flag, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    STS_CK(cudaStreamSynchronize(h->stream));
    if (!flag) return STS_OK;
    STS_CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
    if (h->d_sched) STS_CK(cudaMemsetAsync(h->d_sched, 0, 2 * sizeof(unsigned), h->stream));
    return set_error(STS_ERR_TIMEOUT, "a shared-memory bulk copy did not complete within its time limit; results "
                                      "of the matvecs and applies since the last check are invalid");
}

}  // namespace sts

using namespace sts;

#define STS_GUARD(body)                                                           \
    try {                                                                         \
        body                                                                      \
    } catch (const std::bad_alloc &) {                                            \
        return set_error(STS_ERR_ALLOC, "host allocation failed");                \
    } catch (...) {                                                               \
        return set_error(STS_ERR_INVALID_ARG, "unexpected exception");            \
    }

extern "C" {

const char *sts_last_error(void) { return g_err; }

const char *sts_version(void) { return "sts-gb300 1.0 (sm_103a)"; }

sts_status sts_jac_create(const sts_jac_desc *desc, sts_jac_t *out) {
    NvtxRange nvtx_range("sts_jac_create");
    g_err[0] = 0;
    STS_GUARD(return create_impl(desc, out);)
}

sts_status sts_jac_update_values(sts_jac_t h, const double *S, const double *U, const double *V,
                                 int values_on_host) {
    NvtxRange nvtx_range("sts_jac_update_values");
    if (!h) return set_error(STS_ERR_INVALID_ARG, "sts_jac_update_values: handle is NULL");
    if (!S || (h->n_pairs > 0 && (!U || !V)))
        return set_error(STS_ERR_INVALID_ARG, "sts_jac_update_values: NULL value array");
    STS_GUARD(h->smw.ready = false; h->dense.ready = false; return load_values(h, S, U, V, values_on_host);)
}

sts_status sts_jac_matvec(sts_jac_t h, const double *x, double *y, int trans) {
    NvtxRange nvtx_range("sts_jac_matvec");
    STS_TRY(check_handle(h, x, y, "sts_jac_matvec"));
    if (trans && (!h->has_T || h->rep != STS_REP_FACTORED))
        return set_error(STS_ERR_INVALID_ARG, "sts_jac_matvec: trans = 1 needs a factored handle with enable_transpose");
    const int dir = trans ? 1 : 0;
    STS_GUARD(return with_layout<double>(h, x, y, h->vin, h->vout, [&](const double *a, double *b) {
        return op_matvec64(h, dir, a, b);
    });)
}

sts_status sts_jac_matvec_noalloc(sts_jac_t h, const double *x, double *y, int trans) {
    NvtxRange nvtx_range("sts_jac_matvec_noalloc");
    STS_TRY(check_handle(h, x, y, "sts_jac_matvec_noalloc"));
    if (h->rep != STS_REP_FACTORED)
        return set_error(STS_ERR_INVALID_ARG, "sts_jac_matvec_noalloc: needs the factored representation");
    if (trans && !h->has_T)
        return set_error(STS_ERR_INVALID_ARG, "sts_jac_matvec_noalloc: trans = 1 needs enable_transpose");
    const int dir = trans ? 1 : 0;
    STS_GUARD(return with_layout<double>(h, x, y, h->vin, h->vout, [&](const double *a, double *b) {
        return mv_apply64_noalloc(h, dir, a, b);
    });)
}

sts_status sts_jac_matvec_f32(sts_jac_t h, const float *x, float *y, int trans) {
    NvtxRange nvtx_range("sts_jac_matvec_f32");
    STS_TRY(check_handle(h, x, y, "sts_jac_matvec_f32"));
    if (h->dtype != STS_MIXED) return set_error(STS_ERR_INVALID_ARG, "sts_jac_matvec_f32: handle has no FP32 operators");
    if (trans && !h->has_T) return set_error(STS_ERR_INVALID_ARG, "sts_jac_matvec_f32: no transposed operators");
    const int dir = trans ? 1 : 0;
    STS_GUARD(return with_layout<float>(h, x, y, h->vin32, h->vout32, [&](const float *a, float *b) {
        return mv_apply32(h, dir, a, b, h->c32);
    });)
}

sts_status sts_jac_bjacobi_setup(sts_jac_t h) {
    NvtxRange nvtx_range("sts_jac_bjacobi_setup");
    if (!h) return set_error(STS_ERR_INVALID_ARG, "sts_jac_bjacobi_setup: handle is NULL");
    STS_GUARD(STS_TRY(check_device(h));
              return h->rep == STS_REP_FACTORED ? smw_setup(h) : dense_setup(h);)
}

sts_status sts_jac_bjacobi_apply(sts_jac_t h, const double *x, double *z, int trans) {
    NvtxRange nvtx_range("sts_jac_bjacobi_apply");
    STS_TRY(check_handle(h, x, z, "sts_jac_bjacobi_apply"));
    const bool ready = h->rep == STS_REP_FACTORED ? h->smw.ready : h->dense.ready;
    if (!ready) return set_error(STS_ERR_NOT_SETUP, "sts_jac_bjacobi_apply: call sts_jac_bjacobi_setup first");
    if (trans && (!h->has_T || h->rep != STS_REP_FACTORED))
        return set_error(STS_ERR_INVALID_ARG, "sts_jac_bjacobi_apply: trans = 1 needs enable_transpose");
    const int dir = trans ? 1 : 0;
    STS_GUARD(return with_layout<double>(h, x, z, h->vin, h->vout, [&](const double *a, double *b) {
        return op_apply64(h, dir, a, b);
    });)
}

sts_status sts_jac_bjacobi_apply_f32(sts_jac_t h, const float *x, float *z, int trans) {
    NvtxRange nvtx_range("sts_jac_bjacobi_apply_f32");
    STS_TRY(check_handle(h, x, z, "sts_jac_bjacobi_apply_f32"));
    if (h->dtype != STS_MIXED) return set_error(STS_ERR_INVALID_ARG, "sts_jac_bjacobi_apply_f32: handle has no FP32 operators");
    if (!h->smw.ready) return set_error(STS_ERR_NOT_SETUP, "sts_jac_bjacobi_apply_f32: call sts_jac_bjacobi_setup first");
    if (trans && !h->has_T) return set_error(STS_ERR_INVALID_ARG, "sts_jac_bjacobi_apply_f32: no transposed operators");
    const int dir = trans ? 1 : 0;
    STS_GUARD(return with_layout<float>(h, x, z, h->vin32, h->vout32, [&](const float *a, float *b) {
        return smw_apply32(h, dir, a, b);
    });)
}

sts_status sts_gmres_solve(sts_jac_t h, const double *b, double *x, const sts_gmres_opts *opts,
                           sts_gmres_info *info) {
    NvtxRange nvtx_range("sts_gmres_solve");
    STS_TRY(check_handle(h, b, x, "sts_gmres_solve"));
    STS_GUARD(const sts_status st = gmres(h, b, x, opts, info);
              if (st == STS_OK || st == STS_ERR_NOT_CONVERGED || st == STS_ERR_NUMERIC) STS_TRY(check_device(h));
              return st;)
}

sts_status sts_jac_grad(sts_jac_t h, const double *lambda, const double *x, double *gS, double *gU, double *gV) {
    NvtxRange nvtx_range("sts_jac_grad");
    STS_TRY(check_handle(h, lambda, x, "sts_jac_grad"));
    if (!gS || (h->n_pairs > 0 && (!gU || !gV))) return set_error(STS_ERR_INVALID_ARG, "sts_jac_grad: NULL output");
    if (h->rep != STS_REP_FACTORED || !h->has_T)
        return set_error(STS_ERR_INVALID_ARG, "sts_jac_grad: needs a factored handle with enable_transpose");
    STS_GUARD(return grad(h, lambda, x, gS, gU, gV);)
}

sts_status sts_selftest_bounded_wait(void *stream_) {
    NvtxRange nvtx_range("sts_selftest_bounded_wait");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    int *d_flag = nullptr, flag = 0;
    if (cudaMalloc(&d_flag, sizeof(int)) != cudaSuccess)
        return set_error(STS_ERR_CUDA, "sts_selftest_bounded_wait: cudaMalloc failed");
    cudaError_t e = cudaMemsetAsync(d_flag, 0, sizeof(int), stream);
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, kTile, 0, stream>>>(d_flag);
        STS_LAUNCHED();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cudaFree(d_flag);
    if (e != cudaSuccess) return set_error(STS_ERR_CUDA, "sts_selftest_bounded_wait: %s", cudaGetErrorString(e));
    if (flag != 1) return set_error(STS_ERR_CUDA, "sts_selftest_bounded_wait: the wait did not give up (flag %d)", flag);
    return set_error(STS_ERR_TIMEOUT, "sts_selftest_bounded_wait: the bounded wait gave up as expected");
}

sts_status sts_launch_count(unsigned long long *count) {
    if (!count) return set_error(STS_ERR_INVALID_ARG, "sts_launch_count: count is NULL");
    *count = g_launches.load(std::memory_order_relaxed);
    return STS_OK;
}

sts_status sts_jac_memory(sts_jac_t h, size_t *bytes) {
    if (!h || !bytes) return set_error(STS_ERR_INVALID_ARG, "sts_jac_memory: NULL argument");
    *bytes = h->bytes;
    return STS_OK;
}

sts_status sts_jac_destroy(sts_jac_t h) {
    NvtxRange nvtx_range("sts_jac_destroy");
    if (!h) return STS_OK;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
    return STS_OK;
}

}  // extern "C"
