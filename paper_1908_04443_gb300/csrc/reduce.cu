// Observables reduction: total fluid mass, fluid density extremes (Fig. 11), maximum |u| (the
// spurious-current measure of Fig. 10) and the moments of the interface points used by a Kasa
// circle/sphere fit of the drop (contact angle).  Two launches: per-block partials with warp-shuffle
// tree reductions, then one block combining them.  All sums in double.
#include <cfloat>
#include <cmath>
#include <mutex>

#include "kernels.h"
#include "lattice.cuh"
#include "reduce.h"

namespace lbmwet {

namespace {

constexpr int RB = 256;   // threads per reduction block

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// kind of each of the NRED slots: 0 sum, 1 max, 2 min
__device__ __forceinline__ int slot_kind(int k) { return k == 1 || k == 3 ? 1 : (k == 2 ? 2 : 0); }

__device__ void block_combine(double (&v)[NRED], double* out) {
    __shared__ double sh[RB / 32][NRED];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NRED; ++k) {
        const int kind = slot_kind(k);
        const double r = kind == 0 ? warp_sum(v[k]) : (kind == 1 ? warp_max(v[k]) : warp_min(v[k]));
        if (lane == 0) sh[w][k] = r;
    }
    __syncthreads();
    if (threadIdx.x < NRED) {
        const int k = threadIdx.x;
        const int kind = slot_kind(k);
        double r = sh[0][k];
        for (int i = 1; i < RB / 32; ++i) {
            const double x = sh[i][k];
            r = kind == 0 ? r + x : (kind == 1 ? fmax(r, x) : fmin(r, x));
        }
        out[k] = r;
    }
}

__device__ __forceinline__ void init_slots(double (&v)[NRED]) {
#pragma unroll
    for (int k = 0; k < NRED; ++k) v[k] = 0.0;
    v[1] = -DBL_MAX;   // rho_max
    v[2] = DBL_MAX;    // rho_min
    v[3] = 0.0;        // max |u|^2
}

__device__ __forceinline__ int wrapp(int v, int n) { return v >= n ? v - n : v; }

// A double's bits as an int64 in the same order as the doubles (finite values; -0 below +0): the
// sign-magnitude pattern of a negative value has its magnitude bits flipped.  The map is its own
// inverse.  Comparisons and extremes then run on the integer pipe: the FP64 pipe of this GPU issues
// under 2 operations per clock per SM, and the per-node compares would otherwise bound the pass.
__device__ __forceinline__ long long ord_bits(long long b) { return b ^ ((b >> 63) & 0x7fffffffffffffffLL); }
__device__ __forceinline__ long long ord(double x) { return ord_bits(__double_as_longlong(x)); }

// Block `blk` of `nblk` over one grid: its nodes blk * RB + threadIdx.x + k * nblk * RB, combined into
// partials[blk * NRED ..].
template <int DIM>
__device__ __forceinline__ void partial_block(const double* __restrict__ rho, const double* __restrict__ u,
                                              const uint8_t* __restrict__ type, int nx, int ny, int nz,
                                              double rho_mid, double hx, double hy, double hz, int blk, int nblk,
                                              double* __restrict__ partials) {
    const long long N = (long long)nx * ny * nz;
    double v[NRED];
    init_slots(v);
    // density extremes and the largest |u|^2 as ordered integers (see ord); u^2 >= +0, whose bits
    // are already in order
    long long kmax = ord(-DBL_MAX), kmin = ord(DBL_MAX), ku = 0;
    const long long kmid = ord(rho_mid);
    for (long long g = blk * (long long)RB + threadIdx.x; g < N; g += (long long)nblk * RB) {
        // (32-bit division: a grid holds fewer than 2^31 / 19 nodes)
        const unsigned gu = unsigned(g), q = gu / unsigned(nx);
        const int x = int(gu - q * unsigned(nx));
        const int y = int(q % unsigned(ny)), z = int(q / unsigned(ny));
        // every load of the node and of its +x, +y (, +z) neighbours is issued before any branch, so
        // that they are in flight together rather than one dependent round trip after another (the
        // fields hold values at every node, solid ones included)
        long long gn[DIM];
        gn[0] = g - x + wrapp(x + 1, nx);
        gn[1] = ((long long)z * ny + wrapp(y + 1, ny)) * nx + x;
        if (DIM == 3) gn[DIM - 1] = ((long long)wrapp(z + 1, nz) * ny + y) * nx + x;
        const uint8_t t = type[g];
        const double r = rho[g];
        double uc[DIM], rnb[DIM];
        uint8_t tnb[DIM];
#pragma unroll
        for (int c = 0; c < DIM; ++c) uc[c] = u[(long long)c * N + g];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            tnb[a] = type[gn[a]];
            rnb[a] = rho[gn[a]];
        }
        if (t & T_SOLID) continue;
        const long long kr = ord(r);
        v[0] += r;
        kmax = kr > kmax ? kr : kmax;
        kmin = kr < kmin ? kr : kmin;
        double u2 = 0.0;
#pragma unroll
        for (int c = 0; c < DIM; ++c) u2 += uc[c] * uc[c];
        const long long k2 = __double_as_longlong(u2);
        ku = k2 > ku ? k2 : ku;
        if (t & T_NEARWALL) continue;
        const int side = (kr > kmid) - (kr < kmid);   // sign of r - rho_mid
        if (side == 0) continue;                      // a link from r == rho_mid never straddles
        // links +x, +y (, +z) to a fluid neighbour away from walls whose density straddles rho_mid
#pragma unroll
        for (int axis = 0; axis < DIM; ++axis) {
            if (tnb[axis] & (T_SOLID | T_NEARWALL)) continue;
            const double rn = rnb[axis];
            // the link straddles rho_mid: r - rho_mid and rn - rho_mid of opposite signs
            const long long kn = ord(rn);
            if (!(side > 0 ? kn < kmid : kn > kmid)) continue;
            const double tt = (rho_mid - r) / (rn - r);
            double px = x, py = y, pz = z;
            if (axis == 0) px += tt;
            if (axis == 1) py += tt;
            if (axis == 2) pz += tt;
            // periodic image nearest to the hint, relative to the hint
            double dx = px - hx, dy = py - hy, dz = (DIM == 3) ? pz - hz : 0.0;
            dx -= nx * rint(dx / nx);
            dy -= ny * rint(dy / ny);
            if (DIM == 3) dz -= nz * rint(dz / nz);
            const double r2 = dx * dx + dy * dy + dz * dz;
            v[4] += 1.0;
            v[5] += dx;
            v[6] += dy;
            v[7] += dz;
            v[8] += dx * dx;
            v[9] += dy * dy;
            v[10] += dz * dz;
            v[11] += dx * dy;
            v[12] += dx * dz;
            v[13] += dy * dz;
            v[14] += dx * r2;
            v[15] += dy * r2;
            v[16] += dz * r2;
            v[17] += r2;
        }
    }
    v[1] = __longlong_as_double(ord_bits(kmax));
    v[2] = __longlong_as_double(ord_bits(kmin));
    v[3] = __longlong_as_double(ku);
    block_combine(v, partials + (long long)blk * NRED);
}

template <int DIM>
__global__ void __launch_bounds__(RB) reduce_partial(const double* __restrict__ rho, const double* __restrict__ u,
                                                     const uint8_t* __restrict__ type, int nx, int ny, int nz,
                                                     double rho_mid, double hx, double hy, double hz,
                                                     double* __restrict__ partials) {
    partial_block<DIM>(rho, u, type, nx, ny, nz, rho_mid, hx, hy, hz, blockIdx.x, gridDim.x, partials);
}

// One block combining nparts partials; err (optional): the grid's error word, stored after the NRED
// results
__device__ __forceinline__ void final_block(const double* __restrict__ partials, int nparts, double* __restrict__ out,
                                            const unsigned* __restrict__ err) {
    double v[NRED];
    init_slots(v);
    for (int i = threadIdx.x; i < nparts; i += RB) {
#pragma unroll
        for (int k = 0; k < NRED; ++k) {
            const double x = partials[(long long)i * NRED + k];
            const int kind = slot_kind(k);
            v[k] = kind == 0 ? v[k] + x : (kind == 1 ? fmax(v[k], x) : fmin(v[k], x));
        }
    }
    block_combine(v, out);
    if (err && threadIdx.x == 0) *reinterpret_cast<unsigned*>(out + NRED) = *err;
}

__global__ void __launch_bounds__(RB) reduce_final(const double* __restrict__ partials, int nparts, double* __restrict__ out,
                                                   const unsigned* __restrict__ err = nullptr) {
    final_block(partials, nparts, out, err);
}

// Several grids in one launch: grid k owns blocks [g[k].block0, g[k].block0 + g[k].nblk), which
// cover its nodes exactly as a launch of g[k].nblk blocks of its own would (same sums, same order).
template <int DIM>
__global__ void __launch_bounds__(RB) reduce_partial_grids(const RedGrid* __restrict__ g, int ngrids) {
    int lo = 0, hi = ngrids - 1;
    while (lo < hi) {   // the last grid whose first block is at or before this one
        const int mid = (lo + hi + 1) >> 1;
        if (g[mid].block0 <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const RedGrid& r = g[lo];
    partial_block<DIM>(r.rho, r.u, r.type, r.nx, r.ny, r.nz, r.rho_mid, r.hint[0], r.hint[1], r.hint[2],
                       int(blockIdx.x) - r.block0, r.nblk, r.partials);
}

__global__ void __launch_bounds__(RB) reduce_final_grids(const RedGrid* __restrict__ g) {
    const RedGrid& r = g[blockIdx.x];
    final_block(r.partials, r.nblk, r.out, r.err);
}

// About 8 nodes per thread: each block ends with warp reductions of NRED doubles on the FP64 pipe,
// whose low rate makes one block per 256 nodes cost more than the nodes themselves on small grids.
int n_blocks(long long N) {
    long long b = (N + 8LL * RB - 1) / (8LL * RB);
    const long long cap = 152LL * 8;
    if (b > cap) b = cap;
    return int(b < 1 ? 1 : b);
}

}  // namespace

size_t reduce_partials_size(long long N) { return size_t(n_blocks(N)) * NRED; }

cudaError_t launch_reduce(int dim, const double* rho, const double* u, const uint8_t* type, int nx, int ny, int nz,
                          double rho_mid, const double* hint, double* partials, double* out, cudaStream_t s) {
    const long long N = (long long)nx * ny * nz;
    const int nb = n_blocks(N);
    if (dim == 2)
        reduce_partial<2><<<nb, RB, 0, s>>>(rho, u, type, nx, ny, nz, rho_mid, hint[0], hint[1], hint[2], partials);
    else
        reduce_partial<3><<<nb, RB, 0, s>>>(rho, u, type, nx, ny, nz, rho_mid, hint[0], hint[1], hint[2], partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_final<<<1, RB, 0, s>>>(partials, nb, out);
    return cudaGetLastError();
}

int reduce_blocks(long long N) { return n_blocks(N); }

cudaError_t launch_reduce_grids(int dim, const RedGrid* grids, int ngrids, int total_blocks, cudaStream_t s) {
    if (ngrids < 1) return cudaSuccess;
    if (dim == 2) reduce_partial_grids<2><<<total_blocks, RB, 0, s>>>(grids, ngrids);
    else reduce_partial_grids<3><<<total_blocks, RB, 0, s>>>(grids, ngrids);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_final_grids<<<ngrids, RB, 0, s>>>(grids);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Allocation-free variant of the observables reduction (no counterpart in the paper).
//
// For callers that must not call cudaMalloc - e.g. frameworks that route every device allocation
// through their own allocator and budget, or latency-sensitive loops where cudaMalloc's implicit
// device synchronisation is not acceptable - the same two kernels run with their per-block
// partials and final sums in this file-scope device array instead of handle-owned buffers.
//
// Capacity: STATIC_BLOCKS blocks of STATIC_NODES_PER_BLOCK nodes, i.e. grids of at most
// 4096 * 4096 = 16,777,216 nodes (256^3); larger grids are rejected.  The array (4096 * 18 + 18
// doubles, about 590 KB) is part of the module image, so every GPU that loads this library holds
// it until the process exits.  All calls share it and it keeps the last call's contents; every
// slot is written by the partial kernel before the final kernel reads it, so nothing needs
// clearing between calls.  Calls whose kernels overlap on the GPU (different streams, or
// different handles on one device without ordering) race on the array.
// ---------------------------------------------------------------------------------------------

namespace {

constexpr int STATIC_BLOCKS = 4096;
constexpr long long STATIC_NODES_PER_BLOCK = 4096;

static __device__ __align__(256) double g_static_scratch[STATIC_BLOCKS * NRED + NRED];

constexpr int MAX_DEVICES = 64;
double* g_static_ptr[MAX_DEVICES] = {nullptr};
std::mutex g_static_mutex;

}  // namespace

long long static_reduce_max_nodes() { return STATIC_BLOCKS * STATIC_NODES_PER_BLOCK; }

cudaError_t static_reduce_setup(int device, double** ptr) {
    if (device < 0 || device >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[device]) {
        // host code may not use the symbol itself as an address: ask the runtime for the device
        // address of this device's copy (the device must be current)
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_ptr[device] = static_cast<double*>(p);
    }
    *ptr = g_static_ptr[device];
    return cudaSuccess;
}

cudaError_t launch_reduce_static(int dim, const double* rho, const double* u, const uint8_t* type, int nx, int ny,
                                 int nz, double rho_mid, const double* hint, double* scratch, double* out_host,
                                 cudaStream_t s) {
    const long long N = (long long)nx * ny * nz;
    const long long nb = (N + STATIC_NODES_PER_BLOCK - 1) / STATIC_NODES_PER_BLOCK;
    if (nb < 1 || nb > STATIC_BLOCKS) return cudaErrorInvalidValue;
    double* partials = scratch;
    double* out = scratch + (long long)STATIC_BLOCKS * NRED;
    if (dim == 2)
        reduce_partial<2><<<int(nb), RB, 0, s>>>(rho, u, type, nx, ny, nz, rho_mid, hint[0], hint[1], hint[2], partials);
    else
        reduce_partial<3><<<int(nb), RB, 0, s>>>(rho, u, type, nx, ny, nz, rho_mid, hint[0], hint[1], hint[2], partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_final<<<1, RB, 0, s>>>(partials, int(nb), out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(out_host, out, sizeof(double) * NRED, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

}  // namespace lbmwet
