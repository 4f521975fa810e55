// Internal interface between the C-ABI host code and the CUDA kernels (not part of the ABI).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace lbmwet {

// Everything a step kernel needs, passed by value.  Doubles are converted to the kernel's compute
// precision inside the kernel.
struct DevParams {
    int nx, ny, nz;
    long long N;                 // nodes
    // Distributions f[a][z][y][x] live at a * fs + (z * ny + y) * fp + x: 2D rows are padded to a
    // multiple of 32 nodes (128 bytes in FP32) so that every grid has TMA tensor maps and every row
    // starts a cache line; per-node arrays (types, wall ids, fields) are not padded.
    int fp;                      // row pitch of the distributions (nodes)
    long long fs;                // stride between directions (nodes)
    int eos_kind;                // 0 PR, 1 CS
    double RT, a, b, aphi;       // EOS: R*T, a, b, a*phi(T) (PR)
    double two_over_G, G;        // Eq. 6 and Eq. 5
    double s_e, s_eps, s_q, s_nu, s_pi, s_m;
    double c_e, c_eps;           // consistency coefficients of the e and eps rows
    double rho_l, rho_g, rho_ref;
    double fx, fy, fz;           // body force
    int wall_kind;               // 0 IVD, 1 VD, 2 SF (solid-fluid interaction, Eq. 8)
    double kappa, rho_w_const;
    double Gw;                   // SF adhesion parameter
    const double* kappa_w;       // per wall node (device) or null
    const int* wall_id;          // per node: index into kappa_w (valid at wall nodes)
    const uint8_t* type;         // per node: T_SOLID | T_WALL | T_NEARWALL | T_BULK
    const uint8_t* tile_solid;   // per tile of the step kernel's grid: a solid node within the tile + 3-node halo
    const uint8_t* pair_solid;   // the same per tile of the FP32 pair kernel; null: FP32 steps use the tile kernel
    // D3Q19 FP32 step kernel: 0 the TMA-staged z-march, 1 the z-pair march, 2 the scalar z-march
    int step3;
    const void* ztmap;           // TMA tensor maps of the two 3D FP32 distribution buffers (device, 2 x 128 B)
    const void* zf0;             // the buffer the first map describes
    const struct ZItem* zitems;  // its work list: one item per CTA (see ZItem)
    int nzitems;
    unsigned* err;               // sticky device error flags
};

// One work item of the TMA-staged z-march: the 32 x 8 column (bx, by) over planes z0 .. z1 - 1 (at
// most 39), and whether those planes need the path of chunks holding solids (a solid within 3 nodes
// of the column's cells on a plane within 3 planes of the range).  Columns the march cannot box (the
// ragged ones and grids smaller than a box) come as the z-pair march's 32-plane chunks.
struct ZItem {
    int bx, by, z0, z1, solid;
};

// One instance of a batch: its own grid, buffers and wall parameter; the physics (EOS, rates,
// sigma, limiter bounds, body force, wall scheme) is shared by the batch.
struct BatchInstance {
    int nx, ny, nz, N;
    int fp, fs;                // distribution row pitch and direction stride
    void* f[2];                // the instance's two distribution buffers
    const uint8_t* type;
    const int* wall_id;
    const double* kappa_w;     // per wall node or null (scalar kappa)
    double kappa;
};
// One work item of the batched tile kernel (a tile of an instance) or of the y-march (a run of rows
// y0 .. y1 - 1 of a column block), with everything it needs (one contiguous record, so that a CTA
// fetches the next item with one load per lane).
struct alignas(16) BatchItem {
    int nx, ny, N, x0, y0, solid;   // solid: a solid node lies within the item's box + 3-node halo
    int inst, y1;
    int fp, fs;                     // distribution row pitch and direction stride
    const void* f[2];
    const uint8_t* type;
    const int* wall_id;
    const double* kappa_w;
    double kappa;
    const void* tmap;               // FP32 pair kernel: the instance's two TMA tensor maps (128 bytes
                                    // each, for f[0] and f[1]) or null
};
static_assert(sizeof(BatchItem) % 16 == 0, "BatchItem is copied as 32-bit words or 16-byte chunks");

// Column and chunk of the FP32 D3Q19 step kernels (z-march and z-pair march share the per-chunk
// solid flags); compile-time, chosen by measurement.
#ifndef LBMWET_Z3F_X
#define LBMWET_Z3F_X 32
#define LBMWET_Z3F_Y 4
#define LBMWET_Z3F_Z 32
#define LBMWET_Z3F_MINB 3
#endif

enum Lat { LAT_D2Q9 = 0, LAT_D3Q19 = 1 };
enum Prec { PREC_FP64 = 0, PREC_FP32 = 1 };

// One fused time step fin -> fout (both post-collision states, storage precision).
cudaError_t launch_step(int lat, int prec, const void* fin, void* fout, const DevParams& p, cudaStream_t s);
// Pull + moments + force of the current state: rho (N doubles) and u (d*N doubles) into device
// buffers; either may be null.
cudaError_t launch_fields(int lat, int prec, const void* fin, const DevParams& p, double* rho, double* u,
                          cudaStream_t s);
// f* such that the next pull yields f^eq(rho0, u0) (rho0: N doubles, u0: d*N doubles or null).
cudaError_t launch_init(int lat, int prec, void* fout, const DevParams& p, const double* rho0, const double* u0,
                        cudaStream_t s);
// Post-streaming state as doubles [q][N] (pull of the stored state).
cudaError_t launch_get_state(int lat, int prec, const void* fin, const DevParams& p, double* fpost, cudaStream_t s);
// Stored state from post-streaming doubles [q][N].
cudaError_t launch_set_state(int lat, int prec, void* fout, const DevParams& p, const double* fpost, cudaStream_t s);
// Batched step: a persistent grid of `ctas` CTAs walks the work list (instance, tile) of every
// instance of the batch; each instance reads f[parity] and writes f[parity ^ 1].
cudaError_t launch_step_batched(int lat, int prec, int parity, const DevParams& phys, const BatchInstance* insts,
                                const BatchItem* items, int n_items, int ctas, cudaStream_t s);
// D2Q9 FP32 step with two nodes per thread (packed FP32x2 arithmetic) on 32 x 16 tiles: one
// grid (tile flags p.pair_solid) or a persistent grid of `ctas` CTAs walking (instance, tile) items,
// claimed dynamically through `sched` (two device counters, zero before the first launch; the
// kernel leaves them zero).
cudaError_t launch_pair_step(const void* fin, void* fout, const DevParams& p, cudaStream_t s);
cudaError_t launch_pair_batched(int parity, const DevParams& phys, const BatchItem* items, int n_items, int ctas,
                                unsigned* sched, cudaStream_t s);
void pair_tile_shape(int* tx, int* ty);
// Measured FP64 fused multiply-add rate of the device (GFLOP/s, best of three timed launches of
// independent FMA chains after one warm-up); synchronises the stream.
cudaError_t probe_fp64_rate(cudaStream_t s, double* gflops);
// Launches a kernel whose mbarrier wait cannot complete (bounded by `limit` polls); sets ERR_TIMEOUT
// in *err.
cudaError_t launch_wait_timeout_probe(unsigned* err, unsigned limit, cudaStream_t s);
// Box (x extent, y extent; all 9 directions) of the pair kernel's TMA load: a tile and the cells its
// pulls read, with x starting 4 cells before the tile (a 16-byte boundary).
void pair_box_dims(int* bx, int* by);
int pair_ctas_per_sm();
// D2Q9 y-march step: `ctas` persistent CTAs of ymarch_threads(prec) threads; CTA c walks the runs
// items[begin[c] .. begin[c + 1]), each reading f[parity] of its grid and writing f[parity ^ 1].
cudaError_t launch_ymarch(int prec, int parity, const DevParams& phys, const BatchItem* items, const int* begin,
                          int ctas, cudaStream_t s);
int ymarch_threads(int prec);
int ymarch_ctas_per_sm(int prec);
// D3Q19 z-march step (mode 0: time step, 1: fields) and its tile (x, y, z-chunk).
struct Geo;
cudaError_t launch_step3d(int prec, int mode, const void* fin, void* fout, const Geo& g, const DevParams& p,
                          double* rho, double* u, cudaStream_t s);
void zmarch_tile_shape(int prec, int* tx, int* ty, int* tz);
// D3Q19 FP32 step as a z-pair march (two planes per thread, packed FP32x2 arithmetic); chunk flags
// g.tile_solid per FP32 z-march chunk.
cudaError_t launch_zpair_step(const void* fin, void* fout, const Geo& g, const DevParams& p, cudaStream_t s);
// D3Q19 FP32 step, TMA-staged z-march over 32 x 8 columns of 32-plane chunks (ragged columns and
// small grids take the z-pair march); tmap: the tensor map of fin (dimensions x, y, 19 nz; box
// bx x by x 1, see ztma_box_dims), 128 bytes.
cudaError_t launch_ztma_step(const void* fin, void* fout, const void* tmap, const Geo& g, const DevParams& p,
                             cudaStream_t s);
void ztma_box_dims(int* bx, int* by);
// Work list of the TMA-staged z-march for a grid with solid mask `mask` (host, nx*ny*nz bytes):
// every boxed 32 x 8 column cut along z into runs that need the solid path and runs that do not
// (bulk runs shorter than 8 planes join the solid path), each run cut at the multiples of 32 planes
// (a first or last piece shorter than 8 planes joins its neighbour); the other columns as the z-pair
// march's 32-plane chunks; ordered by first plane, then column.
std::vector<ZItem> ztma_work_list(const uint8_t* mask, int nx, int ny, int nz);
// Tile shape (x, y, z) of the step kernels and the resident CTAs per SM of the batched kernel.
void step_tile_shape(int lat, int prec, int* tx, int* ty, int* tz);
int batched_ctas_per_sm(int lat, int prec);
// Node-type flags from the solid mask: T_SOLID, T_WALL (solid with a fluid lattice neighbour),
// T_NEARWALL (within Euclidean distance 3 of a solid node) and T_BULK (fluid with every lattice
// neighbour fluid).
cudaError_t launch_classify(int lat, const uint8_t* mask, uint8_t* type, int nx, int ny, int nz, cudaStream_t s);
// Per-node wall index map of N nodes: -1 everywhere, then wall_id[idx[i]] = i for the nw wall nodes
// idx (device, ascending linear indices).
cudaError_t launch_wall_ids(const int* idx, int nw, int* wall_id, long long N, cudaStream_t s);

// Observables reduction over rho/u/type: out[0..3] = mass, rho_max, rho_min, max |u|^2;
// out[4..17] = interface-point moments (n, Sx, Sy, Sz, Sxx, Syy, Szz, Sxy, Sxz, Syz, Sx r2, Sy r2,
// Sz r2, S r2) of the points relative to `hint`.  `partials` needs reduce_partials_size() doubles.
constexpr int NRED = 18;
size_t reduce_partials_size(long long N);
cudaError_t launch_reduce(int dim, const double* rho, const double* u, const uint8_t* type, int nx, int ny, int nz,
                          double rho_mid, const double* hint, double* partials, double* out, cudaStream_t s);

// Allocation-free observables reduction: per-block partials and the final sums live in a
// file-scope device array of reduce.cu.  static_reduce_setup() resolves this device's address of
// that array (once per device; the device must be current); launch_reduce_static() runs the
// reduction into it and copies the NRED results to out_host, synchronising the stream.  Grids
// above static_reduce_max_nodes() are refused with cudaErrorInvalidValue.
long long static_reduce_max_nodes();
cudaError_t static_reduce_setup(int device, double** ptr);
cudaError_t launch_reduce_static(int dim, const double* rho, const double* u, const uint8_t* type, int nx, int ny,
                                 int nz, double rho_mid, const double* hint, double* scratch, double* out_host,
                                 cudaStream_t s);

}  // namespace lbmwet
