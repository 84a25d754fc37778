// sts_internal.h -- internal data structures of libsts (not part of the ABI).
//
// Internal layout ("component-major, 32-cell tiles"): cells are grouped in
// tiles of 32 consecutive cells, one cell per lane of a warp.  Every per-cell
// array is stored [...][cell] with the cell index fastest, so that a warp that
// processes one tile reads 32 consecutive values with one coalesced request.
// Internal vectors are x[q * ncp + cell] with ncp = 32 * n_tiles (padding cells
// hold zeros and have no blocks).
//
// On GB300 a warp-wide FP64 FMA occupies an SM sub-partition's FP64 pipe for
// 64 cycles whatever the number of active lanes, so the kernels give every lane
// useful FP64 work (lane = cell), never reduce across lanes in FP64, and keep
// the FP64 instruction count at one FMA per multiply-add of the method.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/sts.h"

namespace sts {

constexpr int kTile = 32;          // cells per tile (one per lane)
constexpr int kMaxSlots = 16;      // block slots per cell (1 diagonal + up to 15 neighbours)
constexpr int kMaxPairsDiag = 16;  // rank-one pairs per diagonal block handled by the SMW setup

// Matvec program descriptor (one per main-stream position):
//   bits 0-15  column q of an S entry, or the pair slot k of a pair term
//   bits 16-20 block slot s of an S entry
//   kDescPair  the position is a pair term u_k[p] * c_k
//   kDescEnd   the row is complete after this position
constexpr unsigned kDescPair = 1u << 29;
constexpr int kPosZero = -2147483647 - 1;     // repack code of a zero (padding) stream position

// Structured pattern family (the paper's StS blocks): the last kStructNF rows
// of a block are dense "flow" rows; a level row p < N = b - kStructNF holds the
// level band |p-q| <= w (w = WD for diagonal blocks, 0 for neighbour blocks)
// and the kStructNF flow columns.  Both S and S^T of such blocks have it.
constexpr int kStructNF = 3;
constexpr int kStructMaxW = 4;
constexpr int kStructMaxSlots = 5;
constexpr unsigned kDescEnd = 1u << 31;

// SMW apply program descriptor (one per stream position):
//   bits 0-11 column j, bits 12-23 row i
//   kApBegin  acc = w_i before this entry (first forward entry of row i)
//   kApScale  acc = value * w_i (the pivot inverse opening backward row i)
//   kApEnd    w_i = acc after this position
constexpr unsigned kApBegin = 1u << 28;
constexpr unsigned kApScale = 1u << 29;
constexpr unsigned kApEnd = 1u << 31;

sts_status set_error(sts_status s, const char *fmt, ...);

#define STS_CK(call)                                                                   \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return ::sts::set_error(STS_ERR_CUDA, "%s failed: %s (%s:%d)", #call,      \
                                    cudaGetErrorString(e_), __FILE__, __LINE__);       \
    } while (0)

// Kernels launched by the library since it was loaded (sts_launch_count).
extern std::atomic<unsigned long long> g_launches;

// After every kernel launch: count it and surface launch errors.
// NVTX range for the life of a scope (visible in Nsight timelines; a no-op
// when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Launch with programmatic dependent launch allowed: the kernel may start
// while the previous kernel on the stream finishes, and must call
// griddepcontrol.wait (pdl_wait) before it reads anything an earlier kernel
// may still write or writes anything an earlier kernel may still read.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

#define STS_LAUNCHED()                                                    \
    do {                                                                  \
        ::sts::g_launches.fetch_add(1, std::memory_order_relaxed);        \
        STS_CK(cudaGetLastError());                                       \
    } while (0)

#define STS_TRY(expr)                    \
    do {                                 \
        sts_status s_ = (expr);          \
        if (s_ != STS_OK) return s_;     \
    } while (0)

// Device allocation tracked by the handle.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// One direction (N: y = J x, T: y = J^T x) of the factored matvec.
//
// Block slots of a cell: slot 0 is the diagonal block; slots 1.. are the
// off-diagonal blocks of the cell's block row (N) or block column (T).
// Pair slots: pairs of slot 0 first (r_diag), then r_off per off-diagonal slot.
// Main stream (per tile, per lane), row by row p = 0..b-1:
//     for s in slots: the values of pattern row p of slot s's kind
//     for k in pair slots: the axpy-vector entry of pair k at row p
// Dot stream: [tile][pair slot][q][lane], the dot-vector of each pair.
// N: S in pattern order, dot-vector V, axpy-vector U, dot input x_col.
// T: S in transposed-pattern order, dot-vector U, axpy-vector V, dot input x_row.
struct MvPlan {
    int n_slots = 0, n_pslots = 0, n_groups = 0;
    int n_dtasks = 0, Lp = 0;                // pass-1 dot tasks per tile, padded dot length
    long long tile_len = 0;                  // main-stream elements per lane per tile
    std::vector<int> h_grp_rows;             // [n_groups+1]
    std::vector<long long> h_row_off;        // [b+1] start of row p in the tile stream
    std::vector<int> h_pslot_slot;           // [n_pslots]
    std::vector<int> h_blk;                  // host copy of blk
    // device copies
    int *nbr = nullptr;                      // [n_tiles][n_slots][32]: input cell or -1
    int *blk = nullptr;                      // [n_tiles][n_slots][32]: public block id or -1
    unsigned *slot_mask = nullptr;           // [n_tiles]: bit s set if any lane has slot s
    int *grp_rows = nullptr;                 // [n_groups+1]
    long long *row_off = nullptr;            // [b+1]
    int *pslot_slot = nullptr;               // [n_pslots]
    int *pslot_local = nullptr;              // [n_pslots]: index of the pair within its block
    int *pat_ptr = nullptr;                  // [2][b+1] pattern rows (kind 0 diag, 1 off), this direction
    int *pat_idx = nullptr;                  // [nnz_d + nnz_o] column indices (kind 1 after kind 0)
    int *pat_src = nullptr;                  // [nnz_d + nnz_o] public entry index of each pattern entry
    int *dtask_slot = nullptr;               // [n_dtasks]: block slot whose x a dot task reads
    int *dpos_kind = nullptr, *dpos_arg = nullptr;   // [n_dtasks*Lp]: pass-1 stream positions
    int *pos_kind = nullptr;                 // [tile_len]: 0..n_slots-1 = S of that slot, -1-k = pair slot k
    int *pos_arg = nullptr;                  // [tile_len]: pattern entry (S) or row p (pair)
    unsigned *desc = nullptr;                // [tile_len]: main-pass program (see kDescPair)
    double *main64 = nullptr;
    float *main32 = nullptr;
    double *dotv64 = nullptr;
    float *dotv32 = nullptr;
    // Dot tasks: the n_pslots pair dots, then (structured layout only) the
    // dense flow rows of S, task n_pslots + f*n_slots + s for flow row N+f of
    // slot s.  Structured main stream, per tile: level rows p < sN (s_rl values
    // each: diagonal band 2*wd+1 (zero-padded where clipped) + NF flow, then per
    // neighbour slot 1 + NF, then the pair terms), then per flow row the
    // n_pslots pair terms.  Warps: n_lgroups groups of s_gl level rows, then one
    // for the flow rows.
    bool structured = false;
    int s_wd = 0, sN = 0, s_rl = 0, s_gl = 0, n_lgroups = 0;
};

// SMW block-Jacobi data (factored representation).
//
// LU pattern = diagonal pattern plus symbolic fill; values stored [slot][cell].
// Apply program (per direction): forward unit-lower sweep, then backward sweep
// "x_i = dinv_i * w_i - sum_j a_ij x_j"; the stream holds the off-diagonal
// coefficients in consumption order.
struct SmwPlan {
    int nnz_lu = 0;
    std::vector<int> h_lu_ptr, h_lu_idx, h_lu_diag;   // CSR of the LU pattern, diagonal slot per row
    std::vector<int> h_src_slot;                      // [nnz_d]: LU slot of each diagonal-pattern entry
    // factorisation schedule
    int *lu_ptr = nullptr, *lu_idx = nullptr, *lu_diag = nullptr;
    int *src_slot = nullptr;
    int *d_ptr = nullptr;                        // diag pattern indptr (row max of S_ii)
    int *f_colL_ptr = nullptr, *f_colL_slot = nullptr;    // L entries of column k: slots (rows > k)
    int *f_upd_ptr = nullptr, *f_upd_tgt = nullptr, *f_upd_src = nullptr;  // per L entry: (i,j) -= l * (k,j)
    int *diag_blk = nullptr;     // [nc] public block id of each cell's diagonal block
    // Apply programs per direction: forward rows i = 0..b-1 and backward rows
    // i = b-1..0 (index r = b-1-i), each a list of (column, LU slot).
    int *ap_fwd_ptr[2] = {nullptr, nullptr}, *ap_fwd_col[2] = {nullptr, nullptr};
    int *ap_bwd_ptr[2] = {nullptr, nullptr}, *ap_bwd_col[2] = {nullptr, nullptr};
    int *ap_fwd_slot[2] = {nullptr, nullptr}, *ap_bwd_slot[2] = {nullptr, nullptr};
    // Stream packing per direction, one entry per stream position: LU slot (or
    // -1 for a pivot inverse) and the row whose pivot inverse scales it (-1: none).
    int *pk_slot[2] = {nullptr, nullptr}, *pk_scale[2] = {nullptr, nullptr};
    unsigned *ap_desc[2] = {nullptr, nullptr};   // apply program (see kApBegin)
    int n_fwd[2] = {0, 0}, n_bwd[2] = {0, 0};
    // per-cell data
    double *Sd = nullptr;        // [nnz_d][ncp] diagonal-block S values
    double *Ud = nullptr;        // [r][b][ncp]
    double *Vd = nullptr;        // [r][b][ncp]
    double *lu = nullptr;        // [nnz_lu][ncp]
    double *dinv = nullptr;      // [b][ncp]
    double *W = nullptr;         // [r][b][ncp]   S^-1 U
    double *Wt = nullptr;        // [r][b][ncp]   S^-T V
    double *Cinv = nullptr;      // [r][r][ncp]   (I + V^T S^-1 U)^-1
    double *ap64[2] = {nullptr, nullptr};   // [n_fwd+n_bwd+b][ncp] apply streams
    float *ap32[2] = {nullptr, nullptr};
    float *W32[2] = {nullptr, nullptr};     // W, Wt rounded
    float *DV32[2] = {nullptr, nullptr};    // Vd, Ud rounded (dot vectors of the two directions)
    int *err_cell = nullptr;     // device: first failing cell (INT_MAX if none)
    bool ready = false;
    // Structured apply (diagonal pattern of the paper's family, no fill): one
    // coefficient stream per direction and precision in ap64 / ap32, s_lt[prec]
    // positions per tile, packed from (spk_src, spk_arg)[prec][dir] (see k_smw_spack).
    bool structured = false;
    int s_w = 0, s_lt[2] = {0, 0};
    int *spk_src[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int *spk_arg[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
};

// Dense-BSR baseline (Section 3.4 storage).
struct DenseRep {
    double *D = nullptr;         // [n_tiles][n_slots][b][b][32]
    double *LU = nullptr;        // [b][b][ncp]
    int *piv = nullptr;          // [b][ncp]
    int *err_cell = nullptr;
    bool ready = false;
};

// GMRES workspace (allocated on first use, grown when needed).
struct Krylov {
    int m = 0;
    double *V = nullptr;         // [m+1][n]
    double *Z = nullptr;         // [m][n]   (flexible or mixed-free FP64 path)
    float *Z32 = nullptr;        // [m][n]   (mixed)
    float *t32a = nullptr, *t32b = nullptr;   // [n]
    double *w = nullptr, *r = nullptr, *xb = nullptr, *bb = nullptr, *tmp = nullptr;  // [n]
    double *partial = nullptr;   // [kRedBlocks][m+2]
    double *red = nullptr;       // [3][m+2] reduced dots and norms
    unsigned int *ticket = nullptr;   // finished-block counter of the last-block reductions (0 between launches)
    double *h_pinned = nullptr;  // host pinned [m+2]
    double *c = nullptr;         // pair dots scratch [n_tiles*n_pslots*32]
    float *c32 = nullptr;
    // A cycle's Arnoldi steps as one CUDA graph (sts_gmres_opts.arnoldi): the
    // Givens state lives on the device, sized for m
    double *gH = nullptr;        // [(m+1) * m] Hessenberg matrix, rotated in place
    double *gcs = nullptr, *gsn = nullptr;   // [m] rotations
    double *gg = nullptr;        // [m+1] rotated right-hand side
    double *ghist = nullptr;     // [m] rotated residual / ||b|| per step
    double *gpar = nullptr;      // [4] stop threshold, history scale, 1 / h(j+1,j), steps allowed
    int *gstate = nullptr;       // [2] steps taken, stop reason (1 criterion met, 2 NaN or Inf)
    double *g_pinned = nullptr;  // host pinned copy of the above
    cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [direction][preconditioned]
    int g_m[2][2] = {{0, 0}, {0, 0}};
    cudaStream_t g_stream[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
};

}  // namespace sts

struct sts_jac_s {
    int nc = 0, b = 0, N = 0, dtype = STS_F64, layout = STS_LAYOUT_CELL_MAJOR;
    int rep = STS_REP_FACTORED;
    int r_diag = 0, r_off = 0, nnz_d = 0, nnz_o = 0, nnzb = 0, n_pairs = 0;
    int n_tiles = 0, ncp = 0;
    bool has_T = false;
    long long nnz_S = 0;
    cudaStream_t stream = nullptr;
    // The last launch of this handle wrote its coefficient streams (values
    // update or block-Jacobi setup): the next hot kernel must not read them
    // before its grid-dependency wait.
    bool streams_dirty = true;
    // launch data computed on first use (per precision: 0 FP64, 1 FP32)
    int device = 0;                     // CUDA device current at creation
    int nsm = 0;                        // SMs of the handle's device
    int l2_bytes = 0;                   // L2 cache of the handle's device
    struct Resident {                   // resident blocks of one structured pass-2 instance
        const void *kern;
        size_t smem;
        int blocks;
    };
    std::vector<Resident> mvs_resident;
    bool sap_attr[2] = {false, false};  // shared-memory limit of the structured apply set
    // host copies of the structure
    std::vector<int> bptr, bidx, dptr, didx, optr, oidx;
    std::vector<long long> soff;    // [nnzb+1]
    std::vector<int> pbase;         // [nnzb+1] pair_indptr
    // device structure
    long long *d_soff = nullptr;
    int *d_pbase = nullptr;
    sts::MvPlan mv[2];
    sts::SmwPlan smw;
    sts::DenseRep dense;
    sts::Krylov kry;
    double *vin = nullptr, *vout = nullptr;     // [b*ncp] layout conversion buffers
    double *staging = nullptr;                  // device copy of host values (first host update on)
    float *vin32 = nullptr, *vout32 = nullptr;
    double *c64 = nullptr;                      // matvec pair dots [n_tiles*n_pslots_max*32]
    int *d_err = nullptr;                       // device: set when a bounded device wait gave up
    unsigned *d_sched = nullptr;                // device: matvec pass-2 item counter, finished warps
    float *c32 = nullptr;
    double *g_c = nullptr;                      // adjoint: pair dots of the T direction
    int *g_pair_cN = nullptr, *g_pair_cT = nullptr, *g_pair_row = nullptr, *g_pair_col = nullptr;
    int *g_blk_row = nullptr, *g_blk_col = nullptr, *g_erow = nullptr;   // erow: [nnz_d + nnz_o]
    std::vector<sts::DevBuf> allocs;
    size_t bytes = 0;
};

namespace sts {

// Band half-width of a pattern of the structured family, or -1 (api.cu).
int struct_band(int b, const std::vector<int> &ptr, const std::vector<int> &idx);

// allocation helpers (api.cu); dev_free releases one tracked allocation
sts_status dev_alloc(sts_jac_s *h, void **p, size_t bytes);
void dev_free(sts_jac_s *h, void *p);
template <typename T>
inline sts_status dalloc(sts_jac_s *h, T **p, size_t n) {
    return dev_alloc(h, reinterpret_cast<void **>(p), n * sizeof(T));
}
template <typename T>
inline sts_status upload(sts_jac_s *h, T **p, const std::vector<T> &v) {
    STS_TRY(dalloc(h, p, v.size() ? v.size() : 1));
    if (!v.empty()) STS_CK(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
    return STS_OK;
}

// kernels_matvec.cu
sts_status mv_repack(sts_jac_s *h, int dir, const double *S, const double *U, const double *V);
sts_status mv_apply64(sts_jac_s *h, int dir, const double *x, double *y, double *c);
sts_status mv_apply32(sts_jac_s *h, int dir, const float *x, float *y, float *c);
sts_status mv_dots64(sts_jac_s *h, int dir, const double *x, double *c);   // pass 1 only
sts_status mv_apply64_noalloc(sts_jac_s *h, int dir, const double *x, double *y);
sts_status to_internal64(sts_jac_s *h, const double *x, double *xi);
sts_status from_internal64(sts_jac_s *h, const double *xi, double *x);
sts_status to_internal32(sts_jac_s *h, const float *x, float *xi);
sts_status from_internal32(sts_jac_s *h, const float *xi, float *x);

// kernels_smw.cu
sts_status smw_build(sts_jac_s *h);                       // host schedule + device tables
sts_status smw_repack(sts_jac_s *h, const double *S, const double *U, const double *V);
sts_status smw_setup(sts_jac_s *h);
sts_status check_device(sts_jac_s *h);                   // STS_ERR_TIMEOUT if a bounded device wait gave up
sts_status smw_apply64(sts_jac_s *h, int dir, const double *x, double *z);
sts_status smw_apply32(sts_jac_s *h, int dir, const float *x, float *z);

// kernels_dense.cu
sts_status dense_build(sts_jac_s *h, const double *S, const double *U, const double *V);
sts_status dense_matvec(sts_jac_s *h, const double *x, double *y);
sts_status dense_setup(sts_jac_s *h);
sts_status dense_apply(sts_jac_s *h, const double *x, double *z);

// kernels_krylov.cu
sts_status op_matvec64(sts_jac_s *h, int dir, const double *x, double *y);
sts_status op_apply64(sts_jac_s *h, int dir, const double *x, double *z);
sts_status gmres(sts_jac_s *h, const double *b, double *x, const sts_gmres_opts *o, sts_gmres_info *info);
sts_status kry_reserve(sts_jac_s *h, int m);
sts_status kry_dots(sts_jac_s *h, const double *V, int k, const double *w, int self, double *out_dev);
sts_status kry_update(sts_jac_s *h, double *w, const double *V, int k, const double *hcoef_dev, int norm,
                      double *out_dev);
sts_status kry_norm2(sts_jac_s *h, const double *v, double *out_dev);
sts_status kry_sub(sts_jac_s *h, double *r, const double *b, const double *y);
sts_status kry_scale(sts_jac_s *h, double *out, const double *in, double s);
sts_status kry_axpy(sts_jac_s *h, double *x, const double *Z, int k, const double *y_dev);

// kernels_grad.cu
sts_status grad(sts_jac_s *h, const double *lam, const double *x, double *gS, double *gU, double *gV);

}  // namespace sts
