// C ABI of lbmwet (see include/lbmwet.h): handle life cycle, the step driver (CUDA-graph chunks of
// fused step kernels), observables, state transfer and checkpoints.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lbmwet.h"
#include "adjoint.h"
#include "eos_host.h"
#include "kernels.h"
#include "lattice.cuh"
#include "maskscan.h"
#include "reduce.h"
#include "plan.h"
#include "wall_gf.h"

using namespace lbmwet;

// NVTX range over one entry point (visible to profilers; no cost without one attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

namespace {

thread_local std::string g_init_error;

constexpr int GRAPH_STEPS = 16;   // steps per captured graph (even: the buffer parity is preserved)

}  // namespace

struct lbm_handle {
    lbm_config cfg{};
    int lat = 0, prec = 0, Q = 9, D = 2;
    long long N = 0;
    cudaStream_t stream = nullptr;
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    size_t fbytes = 0;   // bytes of one distribution buffer
    uint8_t* d_type = nullptr;
    uint8_t* d_tile_solid = nullptr;
    std::vector<uint8_t> tile_solid;   // per step-kernel tile: a solid node within the tile + 3-node halo
    std::vector<uint8_t> pair_solid;   // the same per tile of the FP32 pair kernel (D2Q9)
    uint8_t* d_pair_solid = nullptr;   // set when this handle steps with the pair kernel
    void* d_zmaps = nullptr;           // D3Q19 FP32: TMA tensor maps of f[0] and f[1]
    ZItem* d_zitems = nullptr;         // and the work list of the TMA-staged z-march
    int tiles[3] = {1, 1, 1};
    int int_tile[3] = {1, 1, 1};
    int* d_wall_id = nullptr;
    double* d_kappa = nullptr;
    std::vector<uint8_t> mask;         // host solid mask (D2Q9: planning of y-march runs)
    bool ymarch = false;               // single-grid steps by the y-march kernel
    BatchItem* d_yitems = nullptr;     // its runs and per-CTA ranges
    int* d_ybegin = nullptr;
    int yctas = 0;
    unsigned* d_err = nullptr;
    double* d_rho = nullptr;
    double* d_u = nullptr;
    double* d_partials = nullptr;
    double* d_red = nullptr;
    std::vector<int64_t> wall_nodes;
    double rho_g = 0, rho_l = 0;
    int64_t step = 0;
    int64_t launches = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    cudaStream_t cap_stream = nullptr;
    DevParams dp{};
    std::string err;
    bool batch_member = false;   // owned and stepped by an lbm_batch
    // recorded trajectory for the adjoint: checkpoints of the stored state every rec_every steps
    std::vector<void*> ckpt;
    int64_t rec_steps = 0, rec_every = 0, rec_end_step = -1;
    int rec_end_cur = 0;
};

namespace {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda)
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// TMA tensor map of one FP32 D2Q9 distribution buffer: dimensions (x, y, direction), the pair
// kernel's box.  False where TMA cannot address the buffer (rows not a multiple of 16 bytes).
// f: a distribution buffer with row pitch fp and direction stride fs (nodes; multiples of 4)
bool encode_pair_map(CUtensorMap* m, void* f, int nx, int ny, int fp, long long fs) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc || fp % 4 != 0 || fs % 4 != 0) return false;
    int bx, by;
    pair_box_dims(&bx, &by);
    const cuuint64_t dims[3] = {cuuint64_t(nx), cuuint64_t(ny), 9};
    const cuuint64_t strides[2] = {cuuint64_t(fp) * 4, cuuint64_t(fs) * 4};
    const cuuint32_t box[3] = {cuuint32_t(bx), cuuint32_t(by), 9};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, f, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// TMA tensor map of one FP32 D3Q19 distribution buffer f[a][z][y][x] seen as a 3D tensor
// (x, y, a * nz + z): the box of the TMA-staged z-march (one direction on one plane, bx x by).
// False where TMA cannot address the buffer (rows not a multiple of 16 bytes).
bool encode_z_map(CUtensorMap* m, void* f, int nx, int ny, int nz, int bx, int by) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc || nx % 4 != 0) return false;
    const cuuint64_t dims[3] = {cuuint64_t(nx), cuuint64_t(ny), cuuint64_t(19) * cuuint64_t(nz)};
    const cuuint64_t strides[2] = {cuuint64_t(nx) * 4, cuuint64_t(nx) * cuuint64_t(ny) * 4};
    const cuuint32_t box[3] = {cuuint32_t(bx), cuuint32_t(by), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, f, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

lbm_status fail(lbm_handle* h, lbm_status s, const std::string& msg) {
    if (h) h->err = msg;
    else g_init_error = msg;
    return s;
}

lbm_status cuda_fail(lbm_handle* h, cudaError_t e, const char* what) {
    return fail(h, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, call)                                     \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

bool rate_ok(double s) { return std::isfinite(s) && s > 0.0 && s < 2.0; }

EosHost to_host(const lbm_eos& e) { return EosHost{e.kind, e.a, e.b, e.R, e.T, e.omega}; }

// Device memory of handles and batches comes from one stream-ordered pool per device that keeps
// freed memory for the next allocation (release threshold: unlimited), so that creating and
// destroying grids repeatedly costs neither a mapping of fresh memory nor a device-wide
// synchronisation per buffer (cudaFree has one); lbm_release_cached_memory hands the pool's unused
// memory back to the driver.  Every allocation is checked to start on a 256-byte boundary (TMA
// tensor maps and vector loads rely on it).
std::mutex& pool_mutex() {
    static std::mutex m;
    return m;
}
std::map<int, cudaMemPool_t>& pools() {
    static std::map<int, cudaMemPool_t> p;
    return p;
}

cudaError_t device_pool(cudaMemPool_t* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(pool_mutex());
    auto it = pools().find(dev);
    if (it != pools().end()) {
        *out = it->second;
        return cudaSuccess;
    }
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = ~uint64_t(0);
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
        cudaMemPoolDestroy(pool);
        return e;
    }
    pools()[dev] = pool;
    *out = pool;
    return cudaSuccess;
}

template <class T>
cudaError_t dmalloc(T** p, size_t bytes, cudaStream_t s) {
    cudaMemPool_t pool;
    cudaError_t e = device_pool(&pool);
    if (e != cudaSuccess) return e;
    void* q = nullptr;
    e = cudaMallocFromPoolAsync(&q, bytes ? bytes : 1, pool, s);
    if (e != cudaSuccess) return e;
    if (reinterpret_cast<uintptr_t>(q) % 256) {
        cudaFreeAsync(q, s);
        return cudaErrorInvalidValue;
    }
    *p = static_cast<T*>(q);
    return cudaSuccess;
}

void dfree(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

// Guard zones: the distribution buffers and the observable fields sit between two GUARD-byte
// zones filled with GUARD_BYTE, so that a kernel writing past either end of one of them leaves a
// trace that lbm_check_guards finds (a check that needs no memory checker).  GUARD keeps the
// inner pointer at the allocation's alignment (256 B) for TMA maps and vector loads.
constexpr size_t GUARD = 4096;
constexpr unsigned char GUARD_BYTE = 0xA5;

cudaError_t guarded_malloc(void** p, size_t bytes, cudaStream_t s) {
    char* base = nullptr;
    cudaError_t e = dmalloc(&base, bytes + 2 * GUARD, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(base, GUARD_BYTE, GUARD, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + GUARD + bytes, GUARD_BYTE, GUARD, s);
    if (e != cudaSuccess) {
        dfree(base, s);
        return e;
    }
    *p = base + GUARD;
    return cudaSuccess;
}

void guarded_free(void* p, cudaStream_t s) {
    if (p) dfree(static_cast<char*>(p) - GUARD, s);
}

// (the caller has synchronised the handle's stream: nothing in flight uses these buffers)
void free_all(lbm_handle* h) {
    cudaStream_t s = h->stream;
    for (int i = 0; i < 2; ++i) {
        if (h->graph[i]) cudaGraphExecDestroy(h->graph[i]);
        guarded_free(h->f[i], s);
    }
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    dfree(h->d_zitems, s);
    for (void* q : {(void*)h->d_type, (void*)h->d_tile_solid, (void*)h->d_pair_solid, h->d_zmaps, (void*)h->d_yitems,
                    (void*)h->d_ybegin, (void*)h->d_wall_id, (void*)h->d_kappa, (void*)h->d_err, (void*)h->d_partials,
                    (void*)h->d_red})
        dfree(q, s);
    guarded_free(h->d_rho, s);
    guarded_free(h->d_u, s);
    for (void* c : h->ckpt) dfree(c, s);
    h->ckpt.clear();
}

// Status and message of a nonzero device error word.  A copy that never landed is a device failure,
// not a numerical one.
lbm_status flag_status(unsigned flags, std::string* msg) {
    std::string m = "device flagged:";
    if (flags & ERR_PSI) m += " non-positive square-root argument in Eq. 6;";
    if (flags & ERR_RHO) m += " non-positive or non-finite density;";
    if (flags & ERR_TIMEOUT) m += " a wait for a shared-memory copy gave up;";
    *msg = m;
    return (flags & ERR_TIMEOUT) ? LBM_ERR_CUDA : LBM_ERR_UNSTABLE;
}

lbm_status check_device_error(lbm_handle* h) {
    unsigned flags = 0;
    CK(h, cudaMemcpyAsync(&flags, h->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (flags) {
        std::string m;
        const lbm_status st = flag_status(flags, &m);
        return fail(h, st, m);
    }
    return LBM_OK;
}

lbm_status ensure_obs_buffers(lbm_handle* h) {
    if (!h->d_rho) CK(h, guarded_malloc(reinterpret_cast<void**>(&h->d_rho), sizeof(double) * h->N, h->stream));
    if (!h->d_u) CK(h, guarded_malloc(reinterpret_cast<void**>(&h->d_u), sizeof(double) * h->N * h->D, h->stream));
    if (!h->d_partials) CK(h, dmalloc(&h->d_partials, sizeof(double) * reduce_partials_size(h->N), h->stream));
    if (!h->d_red) CK(h, dmalloc(&h->d_red, sizeof(double) * NRED, h->stream));
    return LBM_OK;
}

cudaError_t launch_handle_step(lbm_handle* h, cudaStream_t s, int from) {
    if (h->ymarch) return launch_ymarch(h->prec, from, h->dp, h->d_yitems, h->d_ybegin, h->yctas, s);
    return launch_step(h->lat, h->prec, h->f[from], h->f[from ^ 1], h->dp, s);
}

lbm_status launch_one_step(lbm_handle* h, cudaStream_t s, int from) {
    cudaError_t e = launch_handle_step(h, s, from);
    if (e != cudaSuccess) return cuda_fail(h, e, "step kernel launch");
    return LBM_OK;
}

lbm_status build_graph(lbm_handle* h, int parity) {
    if (!h->cap_stream) CK(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    int b = parity;
    for (int i = 0; i < GRAPH_STEPS; ++i) {
        cudaError_t e = launch_handle_step(h, h->cap_stream, b);
        if (e != cudaSuccess) {
            cudaStreamEndCapture(h->cap_stream, &g);
            if (g) cudaGraphDestroy(g);
            return cuda_fail(h, e, "graph capture");
        }
        b ^= 1;
    }
    CK(h, cudaStreamEndCapture(h->cap_stream, &g));
    cudaError_t e = cudaGraphInstantiate(&h->graph[parity], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    return LBM_OK;
}

lbm_status enqueue_steps(lbm_handle* h, int64_t n) {
    if (n < 0) return fail(h, LBM_ERR_ARG, "negative step count");
    while (n > 0) {
        if (n >= GRAPH_STEPS) {
            if (!h->graph[h->cur]) {
                lbm_status st = build_graph(h, h->cur);
                if (st != LBM_OK) return st;
            }
            CK(h, cudaGraphLaunch(h->graph[h->cur], h->stream));
            h->launches += GRAPH_STEPS;
            n -= GRAPH_STEPS;
            h->step += GRAPH_STEPS;
        } else {
            lbm_status st = launch_one_step(h, h->stream, h->cur);
            if (st != LBM_OK) return st;
            h->cur ^= 1;
            h->launches += 1;
            n -= 1;
            h->step += 1;
        }
    }
    return LBM_OK;
}

// lbm_obs from the NRED sums of the observables reduction (mass, density extremes, max |u|^2,
// interface-point moments): the Kasa circle/sphere fit and the contact angle on the handle's body.
// Shared by lbm_observables and lbm_observables_noalloc.
void obs_from_reduction(const lbm_handle* h, const double* red, lbm_obs* out) {
    std::memset(out, 0, sizeof(*out));
    out->mass = red[0];
    out->rho_max = red[1];
    out->rho_min = red[2];
    out->u_max = std::sqrt(red[3]);
    out->step = h->step;
    out->theta_deg = NAN;
    out->drop_radius = NAN;
    for (int k = 0; k < 3; ++k) out->drop_center[k] = NAN;
    const double n = red[4];
    out->n_interface = (int64_t)n;
    const int D = h->D;
    if (!(n >= D + 1)) return;
    // Kasa normal equations for (D_1..D_d, F): sum (|p|^2 + D.p + F)^2 minimal, p relative to the hint
    const double m1[3] = {red[5], red[6], red[7]};
    const double mxx[3][3] = {{red[8], red[11], red[12]}, {red[11], red[9], red[13]}, {red[12], red[13], red[10]}};
    const double mr[3] = {red[14], red[15], red[16]};
    const int m = D + 1;
    double A[4][5];
    for (int i = 0; i < D; ++i) {
        for (int j = 0; j < D; ++j) A[i][j] = mxx[i][j];
        A[i][D] = m1[i];
        A[i][m] = -mr[i];
    }
    for (int j = 0; j < D; ++j) A[D][j] = m1[j];
    A[D][D] = n;
    A[D][m] = -red[17];
    for (int col = 0; col < m; ++col) {
        int piv = col;
        for (int r = col + 1; r < m; ++r)
            if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
        if (std::fabs(A[piv][col]) < 1e-300) return;
        for (int j = 0; j <= m; ++j) std::swap(A[col][j], A[piv][j]);
        for (int r = 0; r < m; ++r) {
            if (r == col) continue;
            const double fct = A[r][col] / A[col][col];
            for (int j = col; j <= m; ++j) A[r][j] -= fct * A[col][j];
        }
    }
    double c[3] = {0, 0, 0}, cc = 0;
    for (int k = 0; k < D; ++k) {
        c[k] = -0.5 * A[k][m] / A[k][k];
        cc += c[k] * c[k];
    }
    const double r2 = cc - A[D][m] / A[D][D];
    if (!(r2 > 0)) return;
    const double r = std::sqrt(r2);
    for (int k = 0; k < D; ++k) out->drop_center[k] = h->cfg.drop_hint[k] + c[k];
    out->drop_radius = r;
    double cth = NAN;
    if (h->cfg.body_kind == LBM_BODY_BALL) {
        const double Rw = h->cfg.body_radius + 0.5;
        double d2 = 0;
        for (int k = 0; k < D; ++k) {
            const double dd = out->drop_center[k] - h->cfg.body_center[k];
            d2 += dd * dd;
        }
        cth = (Rw * Rw + r * r - d2) / (2.0 * Rw * r);
    } else if (h->cfg.body_kind == LBM_BODY_PLANE) {
        cth = -(out->drop_center[1] - h->cfg.body_center[1]) / r;
    }
    if (!std::isnan(cth)) {
        cth = cth > 1 ? 1 : (cth < -1 ? -1 : cth);
        out->theta_deg = std::acos(cth) * 180.0 / M_PI;
    }
}


}  // namespace

extern "C" {

const char* lbm_status_string(lbm_status s) {
    switch (s) {
        case LBM_OK: return "ok";
        case LBM_ERR_ARG: return "invalid argument";
        case LBM_ERR_CUDA: return "CUDA error";
        case LBM_ERR_OOM: return "out of device memory";
        case LBM_ERR_UNSTABLE: return "numerically unstable state";
        case LBM_ERR_STATE: return "invalid state";
    }
    return "unknown status";
}

const char* lbm_last_error(const lbm_handle* h) { return h ? h->err.c_str() : g_init_error.c_str(); }

lbm_status lbm_critical_temperature(const lbm_eos* eos, double* tc) {
    if (!eos || !tc) return fail(nullptr, LBM_ERR_ARG, "null argument");
    if (!(eos->a > 0 && eos->b > 0 && eos->R > 0) || (eos->kind != LBM_EOS_PR && eos->kind != LBM_EOS_CS))
        return fail(nullptr, LBM_ERR_ARG, "EOS constants must be positive and the kind PR or CS");
    *tc = critical_temperature(to_host(*eos));
    return LBM_OK;
}

lbm_status lbm_coexistence(const lbm_eos* eos, double* rho_g, double* rho_l) {
    if (!eos || !rho_g || !rho_l) return fail(nullptr, LBM_ERR_ARG, "null argument");
    double tc;
    lbm_status st = lbm_critical_temperature(eos, &tc);
    if (st != LBM_OK) return st;
    if (!(eos->T > 0 && eos->T < tc)) return fail(nullptr, LBM_ERR_ARG, "temperature must be in (0, Tc)");
    if (!coexistence(to_host(*eos), rho_g, rho_l)) return fail(nullptr, LBM_ERR_ARG, "no coexistence found");
    return LBM_OK;
}

namespace {

// The checks of lbm_init on a configuration (no device work).
lbm_status validate_config(const lbm_config& c, const double* kappa_per_wall) {
    if (c.lattice != LBM_D2Q9 && c.lattice != LBM_D3Q19) return fail(nullptr, LBM_ERR_ARG, "unknown lattice");
    if (c.precision != LBM_FP64 && c.precision != LBM_FP32_DEV) return fail(nullptr, LBM_ERR_ARG, "unknown precision");
    if (c.nx < 1 || c.ny < 1 || c.nz < 1) return fail(nullptr, LBM_ERR_ARG, "grid sizes must be >= 1");
    if (c.lattice == LBM_D2Q9 && c.nz != 1) return fail(nullptr, LBM_ERR_ARG, "D2Q9 needs nz = 1");
    const long long N = (long long)c.nx * c.ny * c.nz;
    if (N > (1LL << 31) / 19) return fail(nullptr, LBM_ERR_ARG, "grid too large");
    if (!rate_ok(c.s_e) || !rate_ok(c.s_eps) || !rate_ok(c.s_q) || !rate_ok(c.s_nu) ||
        (c.lattice == LBM_D3Q19 && (!rate_ok(c.s_pi) || !rate_ok(c.s_m))))
        return fail(nullptr, LBM_ERR_ARG, "relaxation rates must lie in (0, 2)");
    if (!(c.G != 0.0) || !std::isfinite(c.G)) return fail(nullptr, LBM_ERR_ARG, "G must be nonzero");
    if (c.wall_kind != LBM_WALL_IVD && c.wall_kind != LBM_WALL_VD && c.wall_kind != LBM_WALL_SF &&
        c.wall_kind != LBM_WALL_GF)
        return fail(nullptr, LBM_ERR_ARG, "unknown wall scheme");
    if (c.wall_kind == LBM_WALL_SF && !std::isfinite(c.Gw)) return fail(nullptr, LBM_ERR_ARG, "Gw must be finite");
    if (c.wall_kind == LBM_WALL_GF) {
        if (c.lattice != LBM_D2Q9)
            return fail(nullptr, LBM_ERR_ARG, "the geometric-formulation scheme is two-dimensional (D2Q9)");
        if (!(c.theta_a > 0.0 && c.theta_a < 180.0))
            return fail(nullptr, LBM_ERR_ARG, "theta_a must lie in (0, 180) degrees");
        if (kappa_per_wall) return fail(nullptr, LBM_ERR_ARG, "kappa_per_wall applies to the IVD scheme");
    }
    if (c.step_kernel != LBM_KERNEL_AUTO && c.step_kernel != LBM_KERNEL_TILE && c.step_kernel != LBM_KERNEL_YMARCH &&
        c.step_kernel != LBM_KERNEL_PAIR && c.step_kernel != LBM_KERNEL_ZTMA)
        return fail(nullptr, LBM_ERR_ARG, "unknown step kernel");
    if (c.step_kernel == LBM_KERNEL_PAIR && c.precision != LBM_FP32_DEV)
        return fail(nullptr, LBM_ERR_ARG, "the pair kernels (D2Q9 pair, D3Q19 z-pair march) are FP32");
    if (c.step_kernel == LBM_KERNEL_YMARCH && c.lattice != LBM_D2Q9)
        return fail(nullptr, LBM_ERR_ARG, "the y-march is a D2Q9 kernel");
    if (c.step_kernel == LBM_KERNEL_ZTMA && (c.lattice != LBM_D3Q19 || c.precision != LBM_FP32_DEV))
        return fail(nullptr, LBM_ERR_ARG, "the TMA-staged z-march is for D3Q19 in FP32");
    double tc;
    lbm_status st = lbm_critical_temperature(&c.eos, &tc);
    if (st != LBM_OK) return st;
    if (!(c.eos.T > 0 && c.eos.T < tc)) return fail(nullptr, LBM_ERR_ARG, "temperature must be in (0, Tc)");
    return LBM_OK;
}

// The mask scan for a validated configuration: the step kernels' tile shape and, for D2Q9 in FP32,
// the pair kernel's.
void scan_for(const lbm_config& c, const uint8_t* solid_mask, int threads, MaskScan* out) {
    int t[3], tp[2];
    step_tile_shape(c.lattice, c.precision, &t[0], &t[1], &t[2]);
    const bool pair = c.lattice == LBM_D2Q9 && c.precision == LBM_FP32_DEV;
    if (pair) pair_tile_shape(&tp[0], &tp[1]);
    scan_mask(solid_mask, c.nx, c.ny, c.nz, c.lattice == LBM_D2Q9 ? 2 : 3, t, pair ? tp : nullptr, threads, out);
}

// lbm_init with the mask scan done by the caller (`pre`, consumed) or here, and with or without the
// closing stream synchronisation (a batch synchronises once for all its members).
lbm_status init_impl(const lbm_config* cfg, const uint8_t* solid_mask, const double* rho0, const double* u0,
                     const double* kappa_per_wall, void* stream, lbm_handle** out, MaskScan* pre, bool sync) {
    if (!cfg || !solid_mask || !out) return fail(nullptr, LBM_ERR_ARG, "null argument");
    *out = nullptr;
    const lbm_config& c = *cfg;
    lbm_status st = validate_config(c, kappa_per_wall);
    if (st != LBM_OK) return st;
    const long long N = (long long)c.nx * c.ny * c.nz;

    lbm_handle* h = new lbm_handle();
    h->cfg = c;
    h->lat = c.lattice;
    h->prec = c.precision;
    h->Q = c.lattice == LBM_D2Q9 ? 9 : 19;
    h->D = c.lattice == LBM_D2Q9 ? 2 : 3;
    h->N = N;
    h->stream = static_cast<cudaStream_t>(stream);
    if (c.rho_l > 0 && c.rho_g > 0) {
        h->rho_g = c.rho_g;
        h->rho_l = c.rho_l;
    } else if (!coexistence(to_host(c.eos), &h->rho_g, &h->rho_l)) {
        delete h;
        return fail(nullptr, LBM_ERR_ARG, "no coexistence densities for this EOS/temperature");
    }
    if (!(h->rho_g < h->rho_l)) {
        delete h;
        return fail(nullptr, LBM_ERR_ARG, "rho_g must be below rho_l");
    }

    // wall nodes (solid nodes with a fluid lattice neighbour, ascending index) and tile flags
    const int nx = c.nx, ny = c.ny, nz = c.nz;
    MaskScan local;
    MaskScan& ms = pre ? *pre : local;
    if (!pre) scan_for(c, solid_mask, scan_threads(N), &ms);
    const long long nfluid = ms.nfluid;
    h->wall_nodes.swap(ms.wall_nodes);
    if (nfluid == 0) {
        delete h;
        return fail(nullptr, LBM_ERR_ARG, "the grid has no fluid node");
    }
    // geometric-formulation scheme: per wall node the crossings of its characteristic lines
    const bool gf = c.wall_kind == LBM_WALL_GF;
    std::vector<double> gf_table;
    if (gf) {
        const size_t nw = h->wall_nodes.size();
        gf_table.assign(GF_STRIDE * (nw ? nw : 1), 0.0);
        std::string msg;
        if (!gf_tables(solid_mask, nx, ny, h->wall_nodes.data(), nw, c.theta_a, gf_table.data(), &msg)) {
            delete h;
            return fail(nullptr, LBM_ERR_ARG, msg);
        }
    }
    // solid flags per tile of the step kernels (see tile_solid_flags)
    {
        int t[3];
        step_tile_shape(c.lattice, c.precision, &t[0], &t[1], &t[2]);
        const int n3[3] = {nx, ny, nz};
        for (int k = 0; k < 3; ++k) {
            h->int_tile[k] = t[k];
            h->tiles[k] = (n3[k] + t[k] - 1) / t[k];
        }
        h->tile_solid.swap(ms.tile_solid);
        h->pair_solid.swap(ms.pair_solid);
    }

    const size_t ssize = c.precision == LBM_FP64 ? sizeof(double) : sizeof(float);
    // distributions: 2D rows padded to a multiple of 32 nodes (128-byte rows in FP32: TMA needs
    // 16-byte row strides, and a row that starts a cache line keeps a warp's 32 consecutive nodes in
    // one line)
    const int fpitch = h->D == 2 ? (nx + 31) / 32 * 32 : nx;
    const long long fstride = (long long)fpitch * ny * nz;
    h->fbytes = ssize * h->Q * (size_t)fstride;
    auto oom = [&](cudaError_t e, const char* what) {
        std::string m = std::string(what) + ": " + cudaGetErrorString(e);
        free_all(h);
        delete h;
        return fail(nullptr, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, m);
    };
    cudaError_t e;
#define CKI(call, what) \
    if ((e = (call)) != cudaSuccess) return oom(e, what)
    CKI(guarded_malloc(&h->f[0], h->fbytes, h->stream), "cudaMalloc f");
    CKI(guarded_malloc(&h->f[1], h->fbytes, h->stream), "cudaMalloc f");
    CKI(dmalloc(&h->d_type, N, h->stream), "cudaMalloc type");
    CKI(dmalloc(&h->d_tile_solid, h->tile_solid.size(), h->stream), "cudaMalloc tile flags");
    CKI(cudaMemcpyAsync(h->d_tile_solid, h->tile_solid.data(), h->tile_solid.size(), cudaMemcpyHostToDevice, h->stream),
        "copy tile flags");
    CKI(dmalloc(&h->d_wall_id, sizeof(int) * N, h->stream), "cudaMalloc wall_id");
    CKI(dmalloc(&h->d_err, sizeof(unsigned), h->stream), "cudaMalloc err");
    const size_t nw = h->wall_nodes.size();
    CKI(dmalloc(&h->d_kappa, sizeof(double) * (gf ? gf_table.size() : (nw ? nw : 1)), h->stream), "cudaMalloc kappa");
    CKI(cudaMemsetAsync(h->d_err, 0, sizeof(unsigned), h->stream), "memset err");
    CKI(cudaMemsetAsync(h->f[0], 0, h->fbytes, h->stream), "memset f");   // padding included
    CKI(cudaMemsetAsync(h->f[1], 0, h->fbytes, h->stream), "memset f");
    {
        // the per-node wall index map, built on the device from the wall list
        const size_t nwl = h->wall_nodes.size();
        std::vector<int32_t> idx(nwl);
        for (size_t i = 0; i < nwl; ++i) idx[i] = int32_t(h->wall_nodes[i]);
        int* d_idx = nullptr;
        if (nwl) {
            CKI(dmalloc(&d_idx, sizeof(int32_t) * nwl, h->stream), "cudaMalloc wall list");
            e = cudaMemcpyAsync(d_idx, idx.data(), sizeof(int32_t) * nwl, cudaMemcpyHostToDevice, h->stream);
            if (e != cudaSuccess) {
                dfree(d_idx, h->stream);
                return oom(e, "copy wall list");
            }
        }
        e = launch_wall_ids(d_idx, int(nwl), h->d_wall_id, N, h->stream);
        dfree(d_idx, h->stream);
        if (e != cudaSuccess) return oom(e, "wall ids");
        if (nwl) h->launches += 1;
    }
    {
        std::vector<double> kap(nw ? nw : 1, c.kappa);
        if (kappa_per_wall)
            for (size_t i = 0; i < nw; ++i) kap[i] = kappa_per_wall[i];
        if (gf) kap.swap(gf_table);
        // (a copy from pageable memory has left the host buffer when the call returns)
        CKI(cudaMemcpyAsync(h->d_kappa, kap.data(), sizeof(double) * kap.size(), cudaMemcpyHostToDevice, h->stream),
            "copy kappa");
    }
    // node classification on the device from the mask (stream-ordered scratch: no device-wide
    // synchronisation for its allocation and release)
    {
        uint8_t* d_mask = nullptr;
        CKI(dmalloc(&d_mask, N, h->stream), "cudaMalloc mask");
        e = cudaMemcpyAsync(d_mask, solid_mask, N, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = launch_classify(h->lat, d_mask, h->d_type, nx, ny, nz, h->stream);
        dfree(d_mask, h->stream);
        if (e != cudaSuccess) return oom(e, "classify");
        h->launches += 1;
    }

    // device parameters
    DevParams& p = h->dp;
    p.nx = nx;
    p.ny = ny;
    p.nz = nz;
    p.N = N;
    p.fp = fpitch;
    p.fs = fstride;
    p.eos_kind = c.eos.kind;
    p.RT = c.eos.R * c.eos.T;
    p.a = c.eos.a;
    p.b = c.eos.b;
    p.aphi = eos_aphi(to_host(c.eos));
    p.G = c.G;
    p.two_over_G = 2.0 / c.G;
    p.s_e = c.s_e;
    p.s_eps = c.s_eps;
    p.s_q = c.s_q;
    p.s_nu = c.s_nu;
    p.s_pi = h->D == 3 ? c.s_pi : 1.0;
    p.s_m = h->D == 3 ? c.s_m : 1.0;
    // consistency coefficients: 12 sigma/(tau - 1/2) in 2D (Eq. 7); 114 and 33 in 3D
    const double ke = h->D == 2 ? 12.0 : 114.0, keps = h->D == 2 ? 12.0 : 33.0;
    p.c_e = ke * c.sigma / (1.0 / c.s_e - 0.5);
    p.c_eps = keps * c.sigma / (1.0 / c.s_eps - 0.5);
    p.rho_l = h->rho_l;
    p.rho_g = h->rho_g;
    p.rho_ref = c.precision == LBM_FP32_DEV ? c.rho_ref : 0.0;
    p.fx = c.body_force[0];
    p.fy = c.body_force[1];
    p.fz = h->D == 3 ? c.body_force[2] : 0.0;
    p.wall_kind = c.wall_kind;
    p.kappa = c.kappa;
    p.rho_w_const = c.rho_w_const;
    p.Gw = c.wall_kind == LBM_WALL_SF ? c.Gw : 0.0;
    p.kappa_w = (kappa_per_wall || gf) ? h->d_kappa : nullptr;   // GF: the crossing tables
    p.wall_id = h->d_wall_id;
    p.type = h->d_type;
    p.tile_solid = h->d_tile_solid;
    p.err = h->d_err;
    // D3Q19 FP32 step kernel and the tensor maps of the TMA-staged z-march
    p.step3 = c.step_kernel == LBM_KERNEL_PAIR ? 1 : (c.step_kernel == LBM_KERNEL_TILE ? 2 : 0);
    p.ztmap = nullptr;
    p.zf0 = h->f[0];
    if (h->D == 3 && c.precision == LBM_FP32_DEV && p.step3 == 0) {
        int bx, by;
        ztma_box_dims(&bx, &by);
        CUtensorMap maps[2];
        if (encode_z_map(&maps[0], h->f[0], nx, ny, nz, bx, by) && encode_z_map(&maps[1], h->f[1], nx, ny, nz, bx, by)) {
            CKI(dmalloc(&h->d_zmaps, sizeof(maps), h->stream), "cudaMalloc tensor maps");
            // (from pageable memory: staged before the call returns, so `maps` may go out of scope)
            CKI(cudaMemcpyAsync(h->d_zmaps, maps, sizeof(maps), cudaMemcpyHostToDevice, h->stream), "copy tensor maps");
            const std::vector<ZItem> items = ztma_work_list(solid_mask, nx, ny, nz);
            CKI(dmalloc(&h->d_zitems, sizeof(ZItem) * items.size(), h->stream), "cudaMalloc work list");
            CKI(cudaMemcpyAsync(h->d_zitems, items.data(), sizeof(ZItem) * items.size(), cudaMemcpyHostToDevice,
                                h->stream), "copy work list");
            p.zitems = h->d_zitems;
            p.nzitems = int(items.size());
            p.ztmap = h->d_zmaps;
        }
    }

    // initial state f = f^eq(rho0, u0), stored so that the first pull yields it
    {
        double* d_rho0 = nullptr;
        double* d_u0 = nullptr;
        CKI(dmalloc(&d_rho0, sizeof(double) * N, h->stream), "cudaMalloc rho0");
        std::vector<double> r0;
        const double* src = rho0;
        if (!rho0) {
            r0.assign(N, h->rho_g);
            src = r0.data();
        }
        e = cudaMemcpyAsync(d_rho0, src, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess && u0) {
            e = dmalloc(&d_u0, sizeof(double) * N * h->D, h->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d_u0, u0, sizeof(double) * N * h->D, cudaMemcpyHostToDevice, h->stream);
        }
        if (e == cudaSuccess) e = launch_init(h->lat, h->prec, h->f[0], p, d_rho0, d_u0, h->stream);
        dfree(d_rho0, h->stream);
        dfree(d_u0, h->stream);
        if (e == cudaSuccess && sync) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return oom(e, "initial state");
        h->launches += 1;
    }
    // D2Q9: keep the mask (batches plan their runs from it); plan this grid's y-march runs if asked
    if (h->D == 2) {
        h->mask.assign(solid_mask, solid_mask + N);
        if (c.step_kernel == LBM_KERNEL_YMARCH) {
            int dev = 0, sms = 1;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            YGrid grid{nx, ny, h->mask.data(), BatchItem{}};
            grid.proto.f[0] = h->f[0];
            grid.proto.f[1] = h->f[1];
            grid.proto.fp = fpitch;
            grid.proto.fs = int(fstride);
            grid.proto.type = h->d_type;
            grid.proto.wall_id = h->d_wall_id;
            grid.proto.kappa_w = h->d_kappa;   // holds the scalar kappa at every wall node unless set per node
            grid.proto.kappa = c.kappa;
            const YPlan plan = plan_ymarch({grid}, ymarch_threads(h->prec), sms * ymarch_ctas_per_sm(h->prec));
            CKI(dmalloc(&h->d_yitems, sizeof(BatchItem) * plan.items.size(), h->stream), "cudaMalloc runs");
            CKI(dmalloc(&h->d_ybegin, sizeof(int) * plan.begin.size(), h->stream), "cudaMalloc runs");
            CKI(cudaMemcpyAsync(h->d_yitems, plan.items.data(), sizeof(BatchItem) * plan.items.size(),
                                cudaMemcpyHostToDevice, h->stream), "copy runs");
            CKI(cudaMemcpyAsync(h->d_ybegin, plan.begin.data(), sizeof(int) * plan.begin.size(),
                                cudaMemcpyHostToDevice, h->stream), "copy runs");
            CKI(cudaStreamSynchronize(h->stream), "sync");
            h->yctas = plan.ctas;
            h->ymarch = true;
        }
        // FP32: the pair kernel unless the tile kernel (or the y-march) was asked for
        if (c.precision == LBM_FP32_DEV && (c.step_kernel == LBM_KERNEL_AUTO || c.step_kernel == LBM_KERNEL_PAIR)) {
            CKI(dmalloc(&h->d_pair_solid, h->pair_solid.size(), h->stream), "cudaMalloc tile flags");
            CKI(cudaMemcpyAsync(h->d_pair_solid, h->pair_solid.data(), h->pair_solid.size(), cudaMemcpyHostToDevice,
                                h->stream),
                "copy tile flags");
            h->dp.pair_solid = h->d_pair_solid;
        }
    }
#undef CKI
    h->cur = 0;
    h->step = 0;
    *out = h;
    return LBM_OK;
}

}  // namespace

lbm_status lbm_init(const lbm_config* cfg, const uint8_t* solid_mask, const double* rho0, const double* u0,
                    const double* kappa_per_wall, void* stream, lbm_handle** out) {
    NvtxRange nvtx_range("lbm_init");
    return init_impl(cfg, solid_mask, rho0, u0, kappa_per_wall, stream, out, nullptr, true);
}

lbm_status lbm_step(lbm_handle* h, int64_t n) {
    NvtxRange nvtx_range("lbm_step");
    if (!h) return LBM_ERR_ARG;
    if (h->batch_member) return fail(h, LBM_ERR_STATE, "a batch member is stepped by lbm_batch_step");
    lbm_status st = enqueue_steps(h, n);
    if (st != LBM_OK) return st;
    CK(h, cudaGetLastError());
    return check_device_error(h);
}

lbm_status lbm_enqueue_steps(lbm_handle* h, int64_t n) {
    NvtxRange nvtx_range("lbm_enqueue_steps");
    if (!h) return LBM_ERR_ARG;
    if (h->batch_member) return fail(h, LBM_ERR_STATE, "a batch member is stepped by lbm_batch_enqueue_steps");
    return enqueue_steps(h, n);
}

lbm_status lbm_check(lbm_handle* h) {
    if (!h) return LBM_ERR_ARG;
    return check_device_error(h);
}

lbm_status lbm_selftest_bounded_wait(void* stream, uint32_t polls, int32_t* timed_out) {
    if (!timed_out || polls == 0) return fail(nullptr, LBM_ERR_ARG, "null argument or zero polls");
    *timed_out = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned* d_flag = nullptr;
    unsigned flag = 0;
    cudaError_t e = dmalloc(&d_flag, sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_flag, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = launch_wait_timeout_probe(d_flag, polls, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, d_flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    dfree(d_flag, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "bounded-wait self-test");
    *timed_out = (flag & ERR_TIMEOUT) ? 1 : 0;
    return LBM_OK;
}

lbm_status lbm_release_cached_memory(void) {
    // frees still pending in streams hold their memory until the streams reach them
    const cudaError_t es = cudaDeviceSynchronize();
    if (es != cudaSuccess) return cuda_fail(nullptr, es, "synchronising before trimming the memory pool");
    std::lock_guard<std::mutex> lock(pool_mutex());
    for (auto& kv : pools()) {
        const cudaError_t e = cudaMemPoolTrimTo(kv.second, 0);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "trimming the device memory pool");
    }
    return LBM_OK;
}

lbm_status lbm_memory_stats(int64_t* reserved_bytes, int64_t* used_bytes) {
    if (!reserved_bytes || !used_bytes) return fail(nullptr, LBM_ERR_ARG, "null argument");
    *reserved_bytes = 0;
    *used_bytes = 0;
    cudaMemPool_t pool;
    cudaError_t e = device_pool(&pool);
    uint64_t r = 0, u = 0;
    if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r);
    if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "memory pool statistics");
    *reserved_bytes = int64_t(r);
    *used_bytes = int64_t(u);
    return LBM_OK;
}

lbm_status lbm_probe_fp64_rate(void* stream, double* gflops) {
    if (!gflops) return fail(nullptr, LBM_ERR_ARG, "null argument");
    *gflops = 0.0;
    cudaError_t e = probe_fp64_rate(static_cast<cudaStream_t>(stream), gflops);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "FP64 rate probe");
    return LBM_OK;
}

lbm_status lbm_check_guards(lbm_handle* h, int64_t* guard_bad, int64_t* pad_bad) {
    if (!h || !guard_bad || !pad_bad) return LBM_ERR_ARG;
    *guard_bad = 0;
    *pad_bad = 0;
    struct Buf {
        const void* p;
        size_t bytes;
    };
    const Buf bufs[4] = {{h->f[0], h->fbytes},
                         {h->f[1], h->fbytes},
                         {h->d_rho, sizeof(double) * (size_t)h->N},
                         {h->d_u, sizeof(double) * (size_t)h->N * h->D}};
    std::vector<unsigned char> zone(2 * GUARD);
    for (const Buf& b : bufs) {
        if (!b.p) continue;
        const char* base = static_cast<const char*>(b.p) - GUARD;
        CK(h, cudaMemcpyAsync(zone.data(), base, GUARD, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaMemcpyAsync(zone.data() + GUARD, base + GUARD + b.bytes, GUARD, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        for (unsigned char v : zone) *guard_bad += v != GUARD_BYTE;
    }
    // padding nodes x in [nx, fp) of every row of both distribution buffers
    const int nx = h->dp.nx, fp = h->dp.fp;
    if (fp > nx) {
        const size_t es = h->prec == LBM_FP64 ? sizeof(double) : sizeof(float);
        const size_t rows = h->fbytes / (es * (size_t)fp);
        std::vector<unsigned char> all(h->fbytes);
        for (int i = 0; i < 2; ++i) {
            CK(h, cudaMemcpyAsync(all.data(), h->f[i], h->fbytes, cudaMemcpyDeviceToHost, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
            for (size_t r = 0; r < rows; ++r)
                for (size_t k = (size_t)nx * es; k < (size_t)fp * es; ++k) *pad_bad += all[r * fp * es + k] != 0;
        }
    }
    return LBM_OK;
}

lbm_status lbm_fields_device(lbm_handle* h, double* rho_dev, double* u_dev) {
    if (!h) return LBM_ERR_ARG;
    cudaError_t e = launch_fields(h->lat, h->prec, h->f[h->cur], h->dp, rho_dev, u_dev, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "fields kernel");
    h->launches += 1;
    return LBM_OK;
}

lbm_status lbm_observables(lbm_handle* h, lbm_obs* out, double* rho_host, double* u_host) {
    NvtxRange nvtx_range("lbm_observables");
    if (!h || !out) return LBM_ERR_ARG;
    lbm_status st = ensure_obs_buffers(h);
    if (st != LBM_OK) return st;
    cudaError_t e = launch_fields(h->lat, h->prec, h->f[h->cur], h->dp, h->d_rho, h->d_u, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "fields kernel");
    const double mid = 0.5 * (h->rho_l + h->rho_g);
    e = launch_reduce(h->D, h->d_rho, h->d_u, h->d_type, h->cfg.nx, h->cfg.ny, h->cfg.nz, mid, h->cfg.drop_hint,
                      h->d_partials, h->d_red, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "reduce kernel");
    h->launches += 3;
    double red[NRED];
    CK(h, cudaMemcpyAsync(red, h->d_red, sizeof(red), cudaMemcpyDeviceToHost, h->stream));
    if (rho_host) CK(h, cudaMemcpyAsync(rho_host, h->d_rho, sizeof(double) * h->N, cudaMemcpyDeviceToHost, h->stream));
    if (u_host)
        CK(h, cudaMemcpyAsync(u_host, h->d_u, sizeof(double) * h->N * h->D, cudaMemcpyDeviceToHost, h->stream));
    st = check_device_error(h);
    if (st != LBM_OK) return st;
    obs_from_reduction(h, red, out);
    return LBM_OK;
}

lbm_status lbm_wall_nodes(const lbm_handle* h, int64_t* idx_out, int64_t* count) {
    if (!h || !count) return LBM_ERR_ARG;
    *count = (int64_t)h->wall_nodes.size();
    if (idx_out)
        for (size_t i = 0; i < h->wall_nodes.size(); ++i) idx_out[i] = h->wall_nodes[i];
    return LBM_OK;
}

lbm_status lbm_get_state(lbm_handle* h, double* f_host) {
    if (!h || !f_host) return LBM_ERR_ARG;
    double* d = nullptr;
    CK(h, dmalloc(&d, sizeof(double) * h->Q * h->N, h->stream));
    cudaError_t e = launch_get_state(h->lat, h->prec, h->f[h->cur], h->dp, d, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f_host, d, sizeof(double) * h->Q * h->N, cudaMemcpyDeviceToHost, h->stream);
    dfree(d, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "get_state");
    h->launches += 1;
    return LBM_OK;
}

lbm_status lbm_set_state(lbm_handle* h, const double* f_host, int64_t step) {
    if (!h || !f_host) return LBM_ERR_ARG;
    double* d = nullptr;
    CK(h, dmalloc(&d, sizeof(double) * h->Q * h->N, h->stream));
    cudaError_t e = cudaMemcpyAsync(d, f_host, sizeof(double) * h->Q * h->N, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = launch_set_state(h->lat, h->prec, h->f[h->cur], h->dp, d, h->stream);
    dfree(d, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_state");
    h->launches += 1;
    h->step = step;
    return LBM_OK;
}

lbm_status lbm_save_state(lbm_handle* h, void* host_buf, size_t* bytes) {
    if (!h || !bytes) return LBM_ERR_ARG;
    const size_t need = h->fbytes + sizeof(int64_t);
    if (!host_buf) {
        *bytes = need;
        return LBM_OK;
    }
    if (*bytes < need) return fail(h, LBM_ERR_ARG, "checkpoint buffer too small");
    CK(h, cudaMemcpyAsync(host_buf, h->f[h->cur], h->fbytes, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    std::memcpy(static_cast<char*>(host_buf) + h->fbytes, &h->step, sizeof(int64_t));
    *bytes = need;
    return LBM_OK;
}

lbm_status lbm_load_state(lbm_handle* h, const void* host_buf, size_t bytes) {
    if (!h || !host_buf) return LBM_ERR_ARG;
    if (bytes != h->fbytes + sizeof(int64_t)) return fail(h, LBM_ERR_ARG, "checkpoint size mismatch");
    CK(h, cudaMemcpyAsync(h->f[h->cur], host_buf, h->fbytes, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    std::memcpy(&h->step, static_cast<const char*>(host_buf) + h->fbytes, sizeof(int64_t));
    return LBM_OK;
}

lbm_status lbm_set_kappa(lbm_handle* h, const double* kappa_per_wall) {
    if (!h || !kappa_per_wall) return LBM_ERR_ARG;
    if (h->cfg.wall_kind != LBM_WALL_IVD) return fail(h, LBM_ERR_ARG, "kappa applies to the IVD scheme");
    const size_t nw = h->wall_nodes.size();
    if (nw) CK(h, cudaMemcpyAsync(h->d_kappa, kappa_per_wall, sizeof(double) * nw, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (!h->dp.kappa_w) {
        // the captured graphs hold the old parameters: rebuild them on next use
        h->dp.kappa_w = h->d_kappa;
        for (int i = 0; i < 2; ++i)
            if (h->graph[i]) {
                cudaGraphExecDestroy(h->graph[i]);
                h->graph[i] = nullptr;
            }
    }
    return LBM_OK;
}

lbm_status lbm_limiter_bounds(const lbm_handle* h, double* rho_g, double* rho_l) {
    if (!h || !rho_g || !rho_l) return LBM_ERR_ARG;
    *rho_g = h->rho_g;
    *rho_l = h->rho_l;
    return LBM_OK;
}

int64_t lbm_kernel_launches(const lbm_handle* h) { return h ? h->launches : 0; }

int32_t lbm_step_kernel_used(const lbm_handle* h) {
    if (!h) return LBM_KERNEL_AUTO;
    if (h->D == 3) {
        if (h->prec == LBM_FP64 || h->dp.step3 == 2) return LBM_KERNEL_TILE;
        return h->dp.step3 == 0 && h->dp.ztmap ? LBM_KERNEL_ZTMA : LBM_KERNEL_PAIR;
    }
    if (h->ymarch) return LBM_KERNEL_YMARCH;
    return h->dp.pair_solid ? LBM_KERNEL_PAIR : LBM_KERNEL_TILE;
}

void lbm_destroy(lbm_handle* h) {
    if (!h || h->batch_member) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    free_all(h);
    delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Allocation-free observables (no counterpart in the paper): see lbm_observables_noalloc in
// include/lbmwet.h.  Reduces caller-provided device fields with the handle's node flags into the
// library's static device scratch; allocates nothing.
// ---------------------------------------------------------------------------------------------


extern "C" lbm_status lbm_observables_noalloc(lbm_handle* h, const double* rho_dev, const double* u_dev,
                                               lbm_obs* out) {
    if (!h || !rho_dev || !u_dev || !out) return fail(h, LBM_ERR_ARG, "null argument");
    if (h->N > static_reduce_max_nodes())
        return fail(h, LBM_ERR_ARG,
                    "grid has " + std::to_string(h->N) + " nodes; the allocation-free reduction's static scratch "
                    "holds at most " + std::to_string(static_reduce_max_nodes()) + " nodes");
    int dev = -1;
    CK(h, cudaGetDevice(&dev));
    double* scratch = nullptr;
    CK(h, static_reduce_setup(dev, &scratch));
    double red[NRED];
    const double mid = 0.5 * (h->rho_l + h->rho_g);
    CK(h, launch_reduce_static(h->D, rho_dev, u_dev, h->d_type, h->cfg.nx, h->cfg.ny, h->cfg.nz, mid,
                               h->cfg.drop_hint, scratch, red, h->stream));
    h->launches += 2;
    obs_from_reduction(h, red, out);
    return LBM_OK;
}

// ---------------------------------------------------------------------------------------------
// Batches: many grids of one physics stepped by one persistent kernel per time step.
// ---------------------------------------------------------------------------------------------

// One group of a batch: the instances stepped by one kernel kind, with its own work list.
struct BatchGroup {
    int kind = LBM_KERNEL_TILE;        // LBM_KERNEL_PAIR, LBM_KERNEL_TILE or LBM_KERNEL_YMARCH
    int ctas_per_sm = 0;               // resident CTAs per SM of its persistent grid (0: the kernel's maximum)
    std::vector<int> members;          // instance indices
    BatchItem* d_items = nullptr;
    int* d_begin = nullptr;            // y-march: per-CTA ranges of d_items
    unsigned* d_sched = nullptr;       // pair kernel: tile-claim counters (zero between launches)
    int n_items = 0, ctas = 1;
    cudaStream_t side = nullptr;       // its branch of the captured steps (batches of several groups)
    cudaEvent_t done = nullptr;
};

struct lbm_batch {
    std::vector<lbm_handle*> inst;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t fork = nullptr;
    int lat = 0, prec = 0, sms = 152, dev = 0;
    DevParams phys{};
    unsigned* d_err = nullptr;
    BatchInstance* d_insts = nullptr;
    void* d_tmaps = nullptr;           // pair kernel: two TMA tensor maps per instance
    std::vector<char> has_map;         // the instance's rows can be addressed by TMA
    std::vector<BatchGroup> groups;
    std::string tuning;                // report of the last lbm_batch_autotune
    int cur = 0;
    int64_t step = 0, launches = 0, nodes = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    std::string err;
    double* h_stage = nullptr;         // pinned: per instance the reduction sums and the error word
    double* d_stage = nullptr;         // the same on the device, filled by the reductions, copied at once
    RedGrid* d_redgrids = nullptr;     // the instances' reduction table (one reduction launch for all)
};

namespace {

lbm_status bfail(lbm_batch* b, lbm_status s, const std::string& msg) {
    if (b) b->err = msg;
    else g_init_error = msg;
    return s;
}

#define CKB(b, call)                                                                                  \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,             \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                         \
    } while (0)

bool same_physics(const lbm_config& a, const lbm_config& b) {
    return a.lattice == b.lattice && a.precision == b.precision && a.eos.kind == b.eos.kind && a.eos.a == b.eos.a &&
           a.eos.b == b.eos.b && a.eos.R == b.eos.R && a.eos.T == b.eos.T && a.eos.omega == b.eos.omega &&
           a.G == b.G && a.sigma == b.sigma && a.s_rho == b.s_rho && a.s_e == b.s_e && a.s_eps == b.s_eps &&
           a.s_j == b.s_j && a.s_q == b.s_q && a.s_nu == b.s_nu && a.s_pi == b.s_pi && a.s_m == b.s_m &&
           a.rho_l == b.rho_l && a.rho_g == b.rho_g && a.rho_ref == b.rho_ref && a.body_force[0] == b.body_force[0] &&
           a.body_force[1] == b.body_force[1] && a.body_force[2] == b.body_force[2] && a.wall_kind == b.wall_kind && a.Gw == b.Gw &&
           a.rho_w_const == b.rho_w_const;
}

// (stream-ordered frees on the batch's stream, behind every launch that reads the lists)
void group_free(BatchGroup& g, cudaStream_t s) {
    dfree(g.d_items, s);
    dfree(g.d_begin, s);
    dfree(g.d_sched, s);
    if (g.side) cudaStreamDestroy(g.side);
    if (g.done) cudaEventDestroy(g.done);
    g.d_items = nullptr;
    g.d_begin = nullptr;
    g.d_sched = nullptr;
    g.side = nullptr;
    g.done = nullptr;
}

void invalidate_graphs(lbm_batch* b) {
    for (int i = 0; i < 2; ++i)
        if (b->graph[i]) {
            cudaGraphExecDestroy(b->graph[i]);
            b->graph[i] = nullptr;
        }
}

void batch_free(lbm_batch* b) {
    invalidate_graphs(b);
    for (BatchGroup& g : b->groups) group_free(g, b->stream);
    b->groups.clear();
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->fork) cudaEventDestroy(b->fork);
    dfree(b->d_err, b->stream);
    dfree(b->d_insts, b->stream);
    dfree(b->d_tmaps, b->stream);
    if (b->h_stage) cudaFreeHost(b->h_stage);
    b->h_stage = nullptr;
    dfree(b->d_stage, b->stream);
    dfree(b->d_redgrids, b->stream);
    for (lbm_handle* h : b->inst) {
        h->batch_member = false;
        lbm_destroy(h);
    }
    b->inst.clear();
}

// Work list of a group: the tiles of its instances (pair kernel: 32 x 16 tiles with the instances'
// TMA maps; tile kernel: its tiles) or the y-march runs planned over its instances; its persistent
// grid of sms x ctas_per_sm CTAs (no more than there are items).
cudaError_t group_build(lbm_batch* b, BatchGroup& g) {
    std::vector<BatchItem> items;
    std::vector<int> begin;
    if (g.kind == LBM_KERNEL_YMARCH) {
        std::vector<YGrid> grids;
        for (int i : g.members) {
            lbm_handle* h = b->inst[i];
            YGrid yg{h->cfg.nx, h->cfg.ny, h->mask.data(), BatchItem{}};
            yg.proto.inst = i;
            yg.proto.f[0] = h->f[0];
            yg.proto.f[1] = h->f[1];
            yg.proto.fp = h->dp.fp;
            yg.proto.fs = int(h->dp.fs);
            yg.proto.type = h->d_type;
            yg.proto.wall_id = h->d_wall_id;
            yg.proto.kappa_w = h->d_kappa;   // per wall node always (holds the scalar kappa unless set)
            yg.proto.kappa = h->dp.kappa;
            grids.push_back(yg);
        }
        const int per_sm = g.ctas_per_sm > 0 ? g.ctas_per_sm : ymarch_ctas_per_sm(b->prec);
        YPlan plan = plan_ymarch(grids, ymarch_threads(b->prec), b->sms * per_sm);
        items = std::move(plan.items);
        begin = std::move(plan.begin);
        g.ctas = plan.ctas;
    } else {
        const bool pair = g.kind == LBM_KERNEL_PAIR;
        int tx, ty, tz;
        step_tile_shape(b->lat, b->prec, &tx, &ty, &tz);
        if (pair) pair_tile_shape(&tx, &ty);
        for (int i : g.members) {
            lbm_handle* h = b->inst[i];
            const int nx = h->cfg.nx, ny = h->cfg.ny;
            for (int y = 0; y < ny; y += ty)
                for (int x = 0; x < nx; x += tx) {
                    const size_t t = (size_t)(y / ty) * ((nx + tx - 1) / tx) + x / tx;
                    BatchItem it{};
                    it.nx = nx;
                    it.ny = ny;
                    it.N = int(h->N);
                    it.fp = h->dp.fp;
                    it.fs = int(h->dp.fs);
                    it.x0 = x;
                    it.y0 = y;
                    it.y1 = std::min(y + ty, ny);
                    it.solid = int(pair ? h->pair_solid[t] : h->tile_solid[t]);
                    it.inst = i;
                    it.f[0] = h->f[0];
                    it.f[1] = h->f[1];
                    it.type = h->d_type;
                    it.wall_id = h->d_wall_id;
                    it.kappa_w = h->d_kappa;   // per wall node always (holds the scalar kappa unless set)
                    it.kappa = h->dp.kappa;
                    it.tmap = pair && b->has_map[i] ? static_cast<const char*>(b->d_tmaps) + 2 * sizeof(CUtensorMap) * i
                                                    : nullptr;
                    items.push_back(it);
                }
        }
        const int max_per_sm = pair ? pair_ctas_per_sm() : batched_ctas_per_sm(b->lat, b->prec);
        const int per_sm = g.ctas_per_sm > 0 && g.ctas_per_sm < max_per_sm ? g.ctas_per_sm : max_per_sm;
        const long long cap = (long long)b->sms * per_sm;
        g.ctas = int((long long)items.size() < cap ? (long long)items.size() : cap);
    }
    g.n_items = int(items.size());
    cudaError_t e = dmalloc(&g.d_items, sizeof(BatchItem) * (items.empty() ? 1 : items.size()), b->stream);
    if (e == cudaSuccess && !items.empty())
        e = cudaMemcpyAsync(g.d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && g.kind == LBM_KERNEL_YMARCH) e = dmalloc(&g.d_begin, sizeof(int) * begin.size(), b->stream);
    if (e == cudaSuccess && g.kind == LBM_KERNEL_YMARCH)
        e = cudaMemcpyAsync(g.d_begin, begin.data(), sizeof(int) * begin.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && g.kind == LBM_KERNEL_PAIR) e = dmalloc(&g.d_sched, 2 * sizeof(unsigned), b->stream);
    if (e == cudaSuccess && g.kind == LBM_KERNEL_PAIR) e = cudaMemsetAsync(g.d_sched, 0, 2 * sizeof(unsigned), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);   // the host item vectors go out of scope
    return e;
}

cudaError_t group_launch(lbm_batch* b, const BatchGroup& g, cudaStream_t s, int parity) {
    if (g.kind == LBM_KERNEL_YMARCH) return launch_ymarch(b->prec, parity, b->phys, g.d_items, g.d_begin, g.ctas, s);
    if (g.kind == LBM_KERNEL_PAIR) return launch_pair_batched(parity, b->phys, g.d_items, g.n_items, g.ctas, g.d_sched, s);
    return launch_step_batched(b->lat, b->prec, parity, b->phys, b->d_insts, g.d_items, g.n_items, g.ctas, s);
}

// One time step of every group: in sequence on s, or (fork) as parallel branches joined back into s
cudaError_t batch_step_groups(lbm_batch* b, cudaStream_t s, int parity, bool fork) {
    if (!fork || b->groups.size() == 1) {
        for (const BatchGroup& g : b->groups) {
            cudaError_t e = group_launch(b, g, s, parity);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    cudaError_t e = cudaEventRecord(b->fork, s);
    for (BatchGroup& g : b->groups) {
        if (e == cudaSuccess) e = cudaStreamWaitEvent(g.side, b->fork, 0);
        if (e == cudaSuccess) e = group_launch(b, g, g.side, parity);
        if (e == cudaSuccess) e = cudaEventRecord(g.done, g.side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, g.done, 0);
    }
    return e;
}

lbm_status batch_launch(lbm_batch* b, cudaStream_t s, int parity) {
    cudaError_t e = batch_step_groups(b, s, parity, false);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("batched step launch: ") + cudaGetErrorString(e));
    return LBM_OK;
}

lbm_status batch_graph(lbm_batch* b, int parity) {
    if (!b->cap_stream) CKB(b, cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    if (b->groups.size() > 1) {
        if (!b->fork) CKB(b, cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
        for (BatchGroup& g : b->groups) {
            if (!g.side) CKB(b, cudaStreamCreateWithFlags(&g.side, cudaStreamNonBlocking));
            if (!g.done) CKB(b, cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming));
        }
    }
    cudaGraph_t graph = nullptr;
    CKB(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    int par = parity;
    for (int i = 0; i < GRAPH_STEPS; ++i) {
        cudaError_t e = batch_step_groups(b, b->cap_stream, par, true);
        if (e != cudaSuccess) {
            cudaStreamEndCapture(b->cap_stream, &graph);
            if (graph) cudaGraphDestroy(graph);
            return bfail(b, LBM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        }
        par ^= 1;
    }
    CKB(b, cudaStreamEndCapture(b->cap_stream, &graph));
    cudaError_t e = cudaGraphInstantiate(&b->graph[parity], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    return LBM_OK;
}

lbm_status batch_enqueue(lbm_batch* b, int64_t n) {
    if (n < 0) return bfail(b, LBM_ERR_ARG, "negative step count");
    const int64_t per_step = (int64_t)b->groups.size();
    while (n > 0) {
        if (n >= GRAPH_STEPS) {
            if (!b->graph[b->cur]) {
                lbm_status st = batch_graph(b, b->cur);
                if (st != LBM_OK) return st;
            }
            CKB(b, cudaGraphLaunch(b->graph[b->cur], b->stream));
            n -= GRAPH_STEPS;
            b->step += GRAPH_STEPS;
            b->launches += GRAPH_STEPS * per_step;
        } else {
            lbm_status st = batch_launch(b, b->stream, b->cur);
            if (st != LBM_OK) return st;
            b->cur ^= 1;
            n -= 1;
            b->step += 1;
            b->launches += per_step;
        }
    }
    for (lbm_handle* h : b->inst) {
        h->cur = b->cur;
        h->step = b->step;
    }
    return LBM_OK;
}

// ---- autotuning of the batch's kernels per grid-size class --------------------------------------

// Size class of an instance: floor(log2(nodes)) (128^2 grids: 14, 512^2: 18).
int size_class(long long nodes) {
    int c = 0;
    while ((2LL << c) <= nodes) ++c;
    return c;
}

struct TuneChoice {
    int kind, ctas_per_sm;
};
// chosen kernels per (device, lattice, precision, size class), shared by every batch of the process
std::map<std::tuple<int, int, int, int>, TuneChoice>& tune_cache() {
    static std::map<std::tuple<int, int, int, int>, TuneChoice> m;
    return m;
}
std::mutex& tune_mutex() {
    static std::mutex m;
    return m;
}

const char* kind_name(int kind) {
    return kind == LBM_KERNEL_PAIR ? "pair" : (kind == LBM_KERNEL_YMARCH ? "ymarch" : "tile");
}

// (Re)build the groups from one choice per instance; instances with the same choice share a group.
lbm_status set_groups(lbm_batch* b, const std::vector<TuneChoice>& choice) {
    invalidate_graphs(b);
    CKB(b, cudaStreamSynchronize(b->stream));
    for (BatchGroup& g : b->groups) group_free(g, b->stream);
    b->groups.clear();
    for (int i = 0; i < (int)b->inst.size(); ++i) {
        BatchGroup* gp = nullptr;
        for (BatchGroup& g : b->groups)
            if (g.kind == choice[i].kind && g.ctas_per_sm == choice[i].ctas_per_sm) gp = &g;
        if (!gp) {
            b->groups.emplace_back();
            gp = &b->groups.back();
            gp->kind = choice[i].kind;
            gp->ctas_per_sm = choice[i].ctas_per_sm;
        }
        gp->members.push_back(i);
    }
    for (BatchGroup& g : b->groups) CKB(b, group_build(b, g));
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_init(int32_t n, const lbm_config* cfgs, const uint8_t* const* masks, const double* const* rho0s,
                          const double* const* kappas_per_wall, void* stream, lbm_batch** out) {
    NvtxRange nvtx_range("lbm_batch_init");
    if (n < 1 || !cfgs || !masks || !out) return bfail(nullptr, LBM_ERR_ARG, "null argument or empty batch");
    *out = nullptr;
    for (int i = 1; i < n; ++i)
        if (!same_physics(cfgs[0], cfgs[i]))
            return bfail(nullptr, LBM_ERR_ARG, "instance " + std::to_string(i) + " differs from instance 0 in lattice, "
                                                "precision or physics (only grid, kappa, body and hint may differ)");
    if (cfgs[0].lattice != LBM_D2Q9) return bfail(nullptr, LBM_ERR_ARG, "batches are implemented for D2Q9");
    const int kernel = cfgs[0].step_kernel;
    if (kernel == LBM_KERNEL_PAIR && cfgs[0].precision != LBM_FP32_DEV)
        return bfail(nullptr, LBM_ERR_ARG, "the pair kernel is for D2Q9 in FP32");
    if (kernel == LBM_KERNEL_ZTMA) return bfail(nullptr, LBM_ERR_ARG, "the TMA-staged z-march is a D3Q19 kernel");
    // host set-up first: every configuration checked, then the members' mask scans spread over the
    // host's cores (one grid per thread), then the device set-up of each member without a
    // synchronisation of its own (one for the batch below)
    for (int i = 0; i < n; ++i) {
        if (!masks[i]) return bfail(nullptr, LBM_ERR_ARG, "instance " + std::to_string(i) + ": null mask");
        lbm_status st = validate_config(cfgs[i], kappas_per_wall ? kappas_per_wall[i] : nullptr);
        if (st != LBM_OK) return bfail(nullptr, st, "instance " + std::to_string(i) + ": " + g_init_error);
    }
    std::vector<MaskScan> scans(n);
    parallel_for(n, int(std::min<unsigned>(16, std::max(1u, std::thread::hardware_concurrency()))),
                 [&](int i) { scan_for(cfgs[i], masks[i], 1, &scans[i]); });
    lbm_batch* b = new lbm_batch();
    b->stream = static_cast<cudaStream_t>(stream);
    b->lat = cfgs[0].lattice;
    b->prec = cfgs[0].precision;
    for (int i = 0; i < n; ++i) {
        lbm_handle* h = nullptr;
        lbm_config ci = cfgs[i];
        ci.step_kernel = LBM_KERNEL_TILE;   // the batch plans its own work; members are not stepped alone
        lbm_status st = init_impl(&ci, masks[i], rho0s ? rho0s[i] : nullptr, nullptr,
                                  kappas_per_wall ? kappas_per_wall[i] : nullptr, stream, &h, &scans[i], false);
        scans[i] = MaskScan();
        if (st != LBM_OK) {
            const std::string m = "instance " + std::to_string(i) + ": " + g_init_error;
            batch_free(b);
            delete b;
            return bfail(nullptr, st, m);
        }
        h->batch_member = true;
        b->inst.push_back(h);
        b->nodes += h->N;
    }
    cudaGetDevice(&b->dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->dev);
    auto setup_fail = [&](cudaError_t e) {
        const std::string m = std::string("batch setup: ") + cudaGetErrorString(e);
        batch_free(b);
        delete b;
        return bfail(nullptr, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, m);
    };
    // instance records of the tile kernel, TMA tensor maps of the pair kernel
    std::vector<BatchInstance> insts(n);
    b->has_map.assign(n, 0);
    std::vector<CUtensorMap> maps(2 * (size_t)n);
    bool any_map = false;
    for (int i = 0; i < n; ++i) {
        lbm_handle* h = b->inst[i];
        BatchInstance& d = insts[i];
        d.nx = h->cfg.nx;
        d.ny = h->cfg.ny;
        d.nz = h->cfg.nz;
        d.N = int(h->N);
        d.fp = h->dp.fp;
        d.fs = int(h->dp.fs);
        d.f[0] = h->f[0];
        d.f[1] = h->f[1];
        d.type = h->d_type;
        d.wall_id = h->d_wall_id;
        d.kappa_w = h->dp.kappa_w;
        d.kappa = h->dp.kappa;
        if (b->prec == LBM_FP32_DEV) {
            b->has_map[i] = encode_pair_map(&maps[2 * i], h->f[0], h->cfg.nx, h->cfg.ny, h->dp.fp, h->dp.fs) &&
                            encode_pair_map(&maps[2 * i + 1], h->f[1], h->cfg.nx, h->cfg.ny, h->dp.fp, h->dp.fs);
            any_map = any_map || b->has_map[i];
        }
    }
    cudaError_t e = dmalloc(&b->d_err, sizeof(unsigned), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(unsigned), b->stream);
    if (e == cudaSuccess) e = dmalloc(&b->d_insts, sizeof(BatchInstance) * n, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_insts, insts.data(), sizeof(BatchInstance) * n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && any_map) e = dmalloc(&b->d_tmaps, sizeof(CUtensorMap) * maps.size(), b->stream);
    if (e == cudaSuccess && any_map)
        e = cudaMemcpyAsync(b->d_tmaps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return setup_fail(e);
    b->phys = b->inst[0]->dp;
    b->phys.err = b->d_err;
    // kernels: the one asked for; with AUTO, the choice an earlier lbm_batch_autotune made for each
    // instance's size class on this device (the pair kernel in FP32, the tile kernel in FP64 where
    // there is none)
    const int dflt = kernel == LBM_KERNEL_AUTO ? (b->prec == LBM_FP32_DEV ? LBM_KERNEL_PAIR : LBM_KERNEL_TILE) : kernel;
    std::vector<TuneChoice> choice(n, TuneChoice{dflt, 0});
    if (kernel == LBM_KERNEL_AUTO) {
        std::lock_guard<std::mutex> lock(tune_mutex());
        for (int i = 0; i < n; ++i) {
            auto it = tune_cache().find(std::make_tuple(b->dev, b->lat, b->prec, size_class(b->inst[i]->N)));
            if (it != tune_cache().end()) choice[i] = it->second;
        }
    }
    lbm_status st = set_groups(b, choice);
    if (st != LBM_OK) {
        const std::string m = b->err;
        batch_free(b);
        delete b;
        return bfail(nullptr, st, m);
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch* b, int32_t trial_steps) {
    NvtxRange nvtx_range("lbm_batch_autotune");
    if (!b) return LBM_ERR_ARG;
    if (trial_steps < 2) return bfail(b, LBM_ERR_ARG, "trial_steps must be at least 2");
    const int trials = trial_steps + (trial_steps & 1);   // even: the state's buffer parity is kept
    const int n = (int)b->inst.size();
    // size classes present and their instances
    std::map<int, std::vector<int>> classes;
    for (int i = 0; i < n; ++i) classes[size_class(b->inst[i]->N)].push_back(i);
    // candidates: the pair kernel at 2, 3 and 4 resident CTAs per SM (FP32), the tile kernel, the
    // y-march
    std::vector<TuneChoice> cand;
    if (b->prec == LBM_FP32_DEV)
        for (int k = pair_ctas_per_sm(); k >= 2; --k) cand.push_back(TuneChoice{LBM_KERNEL_PAIR, k});
    cand.push_back(TuneChoice{LBM_KERNEL_TILE, 0});
    cand.push_back(TuneChoice{LBM_KERNEL_YMARCH, 0});
    CKB(b, cudaStreamSynchronize(b->stream));
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    CKB(b, cudaEventCreate(&t0));
    CKB(b, cudaEventCreate(&t1));
    std::vector<TuneChoice> choice(n, TuneChoice{b->prec == LBM_FP32_DEV ? LBM_KERNEL_PAIR : LBM_KERNEL_TILE, 0});
    std::string report;
    lbm_status result = LBM_OK;
    for (auto& kv : classes) {
        const std::vector<int>& mem = kv.second;
        long long nodes = 0;
        for (int i : mem) nodes += b->inst[i]->N;
        // the members' current state, restored after the trials
        std::vector<void*> saved(mem.size(), nullptr);
        for (size_t k = 0; k < mem.size() && result == LBM_OK; ++k) {
            lbm_handle* h = b->inst[mem[k]];
            cudaError_t e = dmalloc(&saved[k], h->fbytes, b->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(saved[k], h->f[b->cur], h->fbytes, cudaMemcpyDeviceToDevice, b->stream);
            if (e != cudaSuccess) result = bfail(b, LBM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
        }
        // The first candidate is the kernel the batch runs untuned; another one is taken only when it
        // is faster by more than TUNE_MARGIN: a class whose choice differs from the others' forms a
        // group of its own, stepped by a launch of its own, which costs more than a near-tie gains
        // (a class choosing the tile kernel over the pair kernel on a 0.02 % difference made the 96-grid
        // batch 8 % slower).
        constexpr double TUNE_MARGIN = 0.03;
        double best = 1e300, first_ms = 0.0;
        TuneChoice pick = choice[mem[0]], best_c = pick;
        for (const TuneChoice& c : cand) {
            if (result != LBM_OK) break;
            BatchGroup g;
            g.kind = c.kind;
            g.ctas_per_sm = c.ctas_per_sm;
            g.members = mem;
            cudaError_t e = group_build(b, g);
            int par = b->cur;
            for (int k = 0; k < 2 && e == cudaSuccess; ++k, par ^= 1) e = group_launch(b, g, b->stream, par);
            if (e == cudaSuccess) e = cudaEventRecord(t0, b->stream);
            for (int k = 0; k < trials && e == cudaSuccess; ++k, par ^= 1) e = group_launch(b, g, b->stream, par);
            if (e == cudaSuccess) e = cudaEventRecord(t1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(t1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
            group_free(g, b->stream);
            if (e != cudaSuccess) {
                result = bfail(b, LBM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
                break;
            }
            const double per_step = double(ms) / trials;
            char line[200];
            std::snprintf(line, sizeof line, "class 2^%d: %zu instances, %lld nodes, %s x %d per SM: %.5f ms/step (%.1f MLUPS)\n",
                          kv.first, mem.size(), nodes, kind_name(c.kind), c.ctas_per_sm, per_step,
                          nodes / (per_step * 1e3));
            report += line;
            if (&c == &cand[0]) first_ms = per_step;
            if (per_step < best) {
                best = per_step;
                best_c = c;
            }
        }
        pick = (best < (1.0 - TUNE_MARGIN) * first_ms) ? best_c : cand[0];
        // restore the state (the trials ran an even number of steps: the state is in f[cur] again)
        for (size_t k = 0; k < mem.size(); ++k) {
            if (!saved[k]) continue;
            lbm_handle* h = b->inst[mem[k]];
            if (result == LBM_OK) {
                cudaError_t e = cudaMemcpyAsync(h->f[b->cur], saved[k], h->fbytes, cudaMemcpyDeviceToDevice, b->stream);
                if (e != cudaSuccess) result = bfail(b, LBM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
            }
            dfree(saved[k], b->stream);
        }
        if (result != LBM_OK) break;
        for (int i : mem) choice[i] = pick;
        char line[120];
        std::snprintf(line, sizeof line, "class 2^%d: chosen %s x %d per SM\n", kv.first, kind_name(pick.kind),
                      pick.ctas_per_sm);
        report += line;
        std::lock_guard<std::mutex> lock(tune_mutex());
        tune_cache()[std::make_tuple(b->dev, b->lat, b->prec, kv.first)] = pick;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (result != LBM_OK) return result;
    // the trials left their error flags (a fault would have shown in the state): keep them
    b->tuning = report;
    return set_groups(b, choice);
}

const char* lbm_batch_tuning_report(const lbm_batch* b) { return b ? b->tuning.c_str() : ""; }

lbm_status lbm_batch_set_kernels(lbm_batch* b, const int32_t* kinds) {
    if (!b || !kinds) return LBM_ERR_ARG;
    std::vector<TuneChoice> choice(b->inst.size());
    for (size_t i = 0; i < b->inst.size(); ++i) {
        const int k = kinds[i];
        if (k != LBM_KERNEL_TILE && k != LBM_KERNEL_YMARCH && k != LBM_KERNEL_PAIR)
            return bfail(b, LBM_ERR_ARG, "instance " + std::to_string(i) + ": the kernel must be TILE, YMARCH or PAIR");
        if (k == LBM_KERNEL_PAIR && b->prec != LBM_FP32_DEV)
            return bfail(b, LBM_ERR_ARG, "the pair kernel is for FP32");
        choice[i] = TuneChoice{k, 0};
    }
    return set_groups(b, choice);
}

void lbm_batch_autotune_forget(void) {
    std::lock_guard<std::mutex> lock(tune_mutex());
    tune_cache().clear();
}

int32_t lbm_batch_instance_kernel(const lbm_batch* b, int32_t i) {
    if (!b || i < 0 || i >= (int32_t)b->inst.size()) return LBM_KERNEL_AUTO;
    for (const BatchGroup& g : b->groups)
        for (int m : g.members)
            if (m == i) return g.kind;
    return LBM_KERNEL_AUTO;
}

lbm_status lbm_batch_enqueue_steps(lbm_batch* b, int64_t n) {
    NvtxRange nvtx_range("lbm_batch_enqueue_steps");
    if (!b) return LBM_ERR_ARG;
    return batch_enqueue(b, n);
}

lbm_status lbm_batch_step(lbm_batch* b, int64_t n) {
    NvtxRange nvtx_range("lbm_batch_step");
    if (!b) return LBM_ERR_ARG;
    lbm_status st = batch_enqueue(b, n);
    if (st != LBM_OK) return st;
    unsigned flags = 0;
    CKB(b, cudaMemcpyAsync(&flags, b->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream));
    CKB(b, cudaStreamSynchronize(b->stream));
    if (flags & ERR_TIMEOUT) return bfail(b, LBM_ERR_CUDA, "a wait for a shared-memory copy gave up");
    if (flags) return bfail(b, LBM_ERR_UNSTABLE, "device flagged a non-positive square-root argument or density");
    return LBM_OK;
}

lbm_status lbm_batch_observables_fields(lbm_batch* b, lbm_obs* out_n, double* const* rho_hosts,
                                        double* const* u_hosts) {
    NvtxRange nvtx_range("lbm_batch_observables_fields");
    if (!b || !out_n) return LBM_ERR_ARG;
    const size_t n = b->inst.size(), W = NRED + 1;
    if (!b->h_stage)
        CKB(b, cudaHostAlloc(reinterpret_cast<void**>(&b->h_stage), sizeof(double) * W * n, cudaHostAllocDefault));
    if (!b->d_stage) CKB(b, dmalloc(&b->d_stage, sizeof(double) * W * n, b->stream));
    if (!b->d_redgrids) CKB(b, dmalloc(&b->d_redgrids, sizeof(RedGrid) * n, b->stream));
    // every instance's fields pass on the batch's stream, then the reductions of all instances in one
    // pair of launches, each instance's sums and error word into its slot of one device array, one
    // copy of the array, then one synchronisation
    std::vector<RedGrid> tab(n);
    int total = 0;
    for (size_t i = 0; i < n; ++i) {
        lbm_handle* h = b->inst[i];
        lbm_status st = ensure_obs_buffers(h);
        if (st != LBM_OK) return bfail(b, st, "instance " + std::to_string(i) + ": " + h->err);
        CKB(b, launch_fields(h->lat, h->prec, h->f[h->cur], h->dp, h->d_rho, h->d_u, h->stream));
        h->launches += 1;
        RedGrid& r = tab[i];
        r.rho = h->d_rho;
        r.u = h->d_u;
        r.type = h->d_type;
        r.err = h->d_err;
        r.partials = h->d_partials;
        r.out = b->d_stage + W * i;
        r.rho_mid = 0.5 * (h->rho_l + h->rho_g);
        for (int k = 0; k < 3; ++k) r.hint[k] = h->cfg.drop_hint[k];
        r.nx = h->cfg.nx;
        r.ny = h->cfg.ny;
        r.nz = h->cfg.nz;
        r.block0 = total;
        r.nblk = reduce_blocks(h->N);
        total += r.nblk;
    }
    // (from pageable memory: staged before the call returns)
    CKB(b, cudaMemcpyAsync(b->d_redgrids, tab.data(), sizeof(RedGrid) * n, cudaMemcpyHostToDevice, b->stream));
    CKB(b, launch_reduce_grids(b->inst[0]->D, b->d_redgrids, int(n), total, b->stream));
    b->inst[0]->launches += 2;
    for (size_t i = 0; i < n; ++i) {
        lbm_handle* h = b->inst[i];
        if (rho_hosts && rho_hosts[i])
            CKB(b, cudaMemcpyAsync(rho_hosts[i], h->d_rho, sizeof(double) * h->N, cudaMemcpyDeviceToHost, h->stream));
        if (u_hosts && u_hosts[i])
            CKB(b, cudaMemcpyAsync(u_hosts[i], h->d_u, sizeof(double) * h->N * h->D, cudaMemcpyDeviceToHost,
                                   h->stream));
    }
    CKB(b, cudaMemcpyAsync(b->h_stage, b->d_stage, sizeof(double) * W * n, cudaMemcpyDeviceToHost, b->stream));
    CKB(b, cudaStreamSynchronize(b->stream));
    for (size_t i = 0; i < n; ++i) {
        unsigned flags = 0;
        std::memcpy(&flags, b->h_stage + W * i + NRED, sizeof(flags));
        if (flags) {
            std::string m;
            const lbm_status st = flag_status(flags, &m);
            b->inst[i]->err = m;
            return bfail(b, st, "instance " + std::to_string(i) + ": " + m);
        }
        obs_from_reduction(b->inst[i], b->h_stage + W * i, &out_n[i]);
    }
    return LBM_OK;
}

lbm_status lbm_batch_observables(lbm_batch* b, lbm_obs* out_n) {
    return lbm_batch_observables_fields(b, out_n, nullptr, nullptr);
}

lbm_status lbm_grid_shape(const lbm_handle* h, int32_t* shape4) {
    if (!h || !shape4) return LBM_ERR_ARG;
    shape4[0] = h->cfg.nx;
    shape4[1] = h->cfg.ny;
    shape4[2] = h->cfg.nz;
    shape4[3] = h->D;
    return LBM_OK;
}

lbm_status lbm_d3q19_work_list(const uint8_t* solid_mask, int32_t nx, int32_t ny, int32_t nz, int32_t* items,
                               int64_t capacity, int64_t* count) {
    if (!solid_mask || !count) return fail(nullptr, LBM_ERR_ARG, "null argument");
    if (nx < 1 || ny < 1 || nz < 1) return fail(nullptr, LBM_ERR_ARG, "grid sizes must be >= 1");
    if ((long long)nx * ny * nz > (1LL << 31) / 19) return fail(nullptr, LBM_ERR_ARG, "grid too large");
    const std::vector<ZItem> v = ztma_work_list(solid_mask, nx, ny, nz);
    *count = (int64_t)v.size();
    if (!items) return LBM_OK;
    if (capacity < (int64_t)v.size()) return fail(nullptr, LBM_ERR_ARG, "capacity below the item count");
    for (size_t i = 0; i < v.size(); ++i) {
        int32_t* o = items + 5 * i;
        o[0] = v[i].bx;
        o[1] = v[i].by;
        o[2] = v[i].z0;
        o[3] = v[i].z1;
        o[4] = v[i].solid;
    }
    return LBM_OK;
}

lbm_handle* lbm_batch_handle(lbm_batch* b, int32_t i) {
    if (!b || i < 0 || i >= (int32_t)b->inst.size()) return nullptr;
    return b->inst[i];
}

int32_t lbm_batch_size(const lbm_batch* b) { return b ? (int32_t)b->inst.size() : 0; }

int64_t lbm_batch_kernel_launches(const lbm_batch* b) { return b ? b->launches : 0; }

int32_t lbm_batch_step_kernel_used(const lbm_batch* b) {
    if (!b || b->groups.empty()) return LBM_KERNEL_AUTO;
    for (const BatchGroup& g : b->groups)
        if (g.kind != b->groups[0].kind) return LBM_KERNEL_AUTO;   // mixed kernels
    return b->groups[0].kind;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : g_init_error.c_str(); }

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    batch_free(b);
    delete b;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Adjoint (D2Q9): gradient of a loss of the final density with respect to per-wall-node kappa.
// ---------------------------------------------------------------------------------------------

extern "C" lbm_status lbm_record(lbm_handle* h, int64_t n_steps, int64_t ckpt_every) {
    NvtxRange nvtx_range("lbm_record");
    if (!h) return LBM_ERR_ARG;
    if (h->batch_member) return fail(h, LBM_ERR_STATE, "a batch member is stepped by lbm_batch_step");
    if (h->D != 2) return fail(h, LBM_ERR_ARG, "the adjoint is implemented for D2Q9");
    if (n_steps < 1 || ckpt_every < 1) return fail(h, LBM_ERR_ARG, "n_steps and ckpt_every must be >= 1");
    if (h->cfg.wall_kind != LBM_WALL_IVD) return fail(h, LBM_ERR_ARG, "the adjoint differentiates the IVD scheme");
    if (!h->dp.kappa_w || h->ymarch) {
        // switch to per-wall-node kappa (d_kappa already holds the scalar value at every wall node)
        // and to the tile kernel, which the adjoint's replay of the recorded segments uses too
        h->dp.kappa_w = h->d_kappa;
        h->ymarch = false;
        for (int i = 0; i < 2; ++i)
            if (h->graph[i]) {
                cudaGraphExecDestroy(h->graph[i]);
                h->graph[i] = nullptr;
            }
    }
    for (void* c : h->ckpt) dfree(c, h->stream);
    h->ckpt.clear();
    h->rec_steps = 0;
    const int64_t nck = (n_steps + ckpt_every - 1) / ckpt_every;
    for (int64_t c = 0; c < nck; ++c) {
        void* buf = nullptr;
        CK(h, dmalloc(&buf, h->fbytes, h->stream));
        h->ckpt.push_back(buf);
        CK(h, cudaMemcpyAsync(buf, h->f[h->cur], h->fbytes, cudaMemcpyDeviceToDevice, h->stream));
        const int64_t len = std::min(ckpt_every, n_steps - c * ckpt_every);
        lbm_status st = enqueue_steps(h, len);
        if (st != LBM_OK) return st;
    }
    h->rec_steps = n_steps;
    h->rec_every = ckpt_every;
    h->rec_end_step = h->step;
    h->rec_end_cur = h->cur;
    return check_device_error(h);
}

extern "C" lbm_status lbm_adjoint(lbm_handle* h, const double* drho_final_dev, double* dkappa_host) {
    NvtxRange nvtx_range("lbm_adjoint");
    if (!h || !drho_final_dev || !dkappa_host) return fail(h, LBM_ERR_ARG, "null argument");
    if (h->rec_steps < 1 || h->step != h->rec_end_step || h->cur != h->rec_end_cur)
        return fail(h, LBM_ERR_STATE, "lbm_adjoint needs an lbm_record whose final state is the current one");
    const size_t nw = h->wall_nodes.size();
    const int64_t every = h->rec_every, n = h->rec_steps;
    const int64_t nck = (int64_t)h->ckpt.size();
    const size_t es = h->prec == LBM_FP64 ? sizeof(double) : sizeof(float);
    // Two segment buffers: slot 0 of a buffer receives a copy of a segment's checkpoint, slots 1.. the
    // recomputed states.  Pass t reverses segment nck - t (recomputed by pass t - 1) and, on a second
    // branch of the same CUDA graph, recomputes segment nck - 1 - t into the other buffer: the two
    // branches share no data, so the recomputation hides behind the latency-bound reverse kernels.
    // The checkpoint copy is issued before the graph, which therefore depends only on the two segment
    // lengths, the adjoint-buffer parity and the buffer index, and is reused across passes.
    void* seg[2] = {nullptr, nullptr};
    void* mu[2] = {nullptr, nullptr};
    void* scratch = nullptr;
    double* dk = nullptr;
    cudaStream_t cap = nullptr, cap2 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    struct Key {
        int64_t rev_len, rec_len;
        int par, rec_buf;
    };
    std::vector<std::pair<Key, cudaGraphExec_t>> graphs;
    lbm_status st = LBM_OK;
    cudaError_t e = cudaMalloc(&seg[0], h->fbytes * (size_t)every);
    if (e == cudaSuccess && nck > 1) e = cudaMalloc(&seg[1], h->fbytes * (size_t)every);
    if (e == cudaSuccess) e = cudaMalloc(&mu[0], h->fbytes);
    if (e == cudaSuccess) e = cudaMalloc(&mu[1], h->fbytes);
    if (e == cudaSuccess) e = cudaMalloc(&scratch, es * adjoint_scratch_elems(h->N));
    if (e == cudaSuccess) e = cudaMalloc(&dk, sizeof(double) * (nw ? nw : 1));
    if (e == cudaSuccess) e = cudaMemsetAsync(dk, 0, sizeof(double) * (nw ? nw : 1), h->stream);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
    AdjointScratch w{scratch};
    int cur = 0;
    if (e == cudaSuccess) e = launch_adjoint_final(h->prec, drho_final_dev, mu[cur], h->dp, h->stream);
    auto slot = [&](int b, int64_t i) {
        return static_cast<void*>(static_cast<char*>(seg[b]) + (size_t)i * h->fbytes);
    };
    auto seg_len = [&](int64_t c) { return c >= 0 && c < nck ? std::min(every, n - c * every) : int64_t(0); };
    // one graph: reverse rev_len steps in buffer rec_buf ^ 1 || recompute rec_len - 1 steps in rec_buf
    auto capture = [&](const Key& k, cudaGraphExec_t* ex) -> cudaError_t {
        cudaGraph_t g = nullptr;
        cudaError_t r0 = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (r0 != cudaSuccess) return r0;
        cudaError_t r = cudaEventRecord(fork, cap);
        if (r == cudaSuccess) r = cudaStreamWaitEvent(cap2, fork, 0);
        for (int64_t i = 0; i + 1 < k.rec_len && r == cudaSuccess; ++i)
            r = launch_step(h->lat, h->prec, slot(k.rec_buf, i), slot(k.rec_buf, i + 1), h->dp, cap2);
        int c2 = k.par;
        for (int64_t i = k.rev_len - 1; i >= 0 && r == cudaSuccess; --i) {
            r = launch_adjoint_step(h->prec, slot(k.rec_buf ^ 1, i), mu[c2], mu[c2 ^ 1], h->dp, w, dk, cap);
            c2 ^= 1;
        }
        if (r == cudaSuccess) r = cudaEventRecord(join, cap2);
        if (r == cudaSuccess) r = cudaStreamWaitEvent(cap, join, 0);
        cudaError_t r1 = cudaStreamEndCapture(cap, &g);
        if (r == cudaSuccess) r = r1;
        if (r == cudaSuccess) r = cudaGraphInstantiate(ex, g, 0);
        if (g) cudaGraphDestroy(g);
        return r;
    };
    for (int64_t t = 0; t <= nck && e == cudaSuccess; ++t) {
        // the buffer of pass t's recomputation; with one segment only buffer 0 exists and t = 1 only reverses
        const Key k{seg_len(nck - t), seg_len(nck - 1 - t), cur, int(t & 1)};
        if (k.rec_len > 0)
            e = cudaMemcpyAsync(slot(k.rec_buf, 0), h->ckpt[nck - 1 - t], h->fbytes, cudaMemcpyDeviceToDevice,
                                h->stream);
        if (e != cudaSuccess) break;
        cudaGraphExec_t ex = nullptr;
        for (auto& kv : graphs)
            if (kv.first.rev_len == k.rev_len && kv.first.rec_len == k.rec_len && kv.first.par == k.par &&
                kv.first.rec_buf == k.rec_buf)
                ex = kv.second;
        if (!ex) {
            e = capture(k, &ex);
            if (e != cudaSuccess) break;
            graphs.push_back({k, ex});
        }
        e = cudaGraphLaunch(ex, h->stream);
        if (k.rev_len % 2) cur ^= 1;
        h->launches += (k.rec_len > 0 ? k.rec_len - 1 : 0) + 2 * k.rev_len;
    }
    if (e == cudaSuccess && nw)
        e = cudaMemcpyAsync(dkappa_host, dk, sizeof(double) * nw, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) st = cuda_fail(h, e, "adjoint");
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    if (cap) cudaStreamDestroy(cap);
    if (cap2) cudaStreamDestroy(cap2);
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    cudaFree(seg[0]);
    cudaFree(seg[1]);
    cudaFree(mu[0]);
    cudaFree(mu[1]);
    cudaFree(scratch);
    cudaFree(dk);
    if (st != LBM_OK) return st;
    return check_device_error(h);
}
