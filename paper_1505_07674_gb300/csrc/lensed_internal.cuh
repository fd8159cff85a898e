// Internal declarations shared by the translation units of the CUDA library.
// Nothing here is part of the C ABI (include/lensed.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lensed.h"

namespace lensed {

// Packed per-component constants, FP32 and FP64 copies, kNC values each.
// The FP32 copy carries, for the constants a coherent rounding error would
// bias (the SIE prefactor, axis ratio, eccentricity and orientation; the
// light profiles' scale, exponent and amplitude), a second float with the
// rounding residual (value - (float)value), used in compensated multiply-
// adds; the FP64 copy has zeros there.
constexpr int kNC = 24;
// Tile of the PSF / chi^2 kernel: kTileW columns x kTileH rows of outputs,
// kPsfThreads threads, each computing kOutPerThread consecutive columns.
constexpr int kTileW = 64;
constexpr int kTileH = 32;
constexpr int kOutPerThread = 8;
constexpr int kPsfThreads = (kTileW / kOutPerThread) * kTileH;  // 256

// Light-profile kinds inside the packed constants.
constexpr int kKindPower = 0;  // Sersic / de Vaucouleurs: 2^-(2^(p2 lg2 R^2 + lc))
constexpr int kKindGauss = 1;  // Gaussian: 2^-(k R^2)
constexpr int kKindFlat = 2;   // flat sky: the constant A
// Device plane of a foreground light component whose parameters are all
// fixed: its pixel integral is the same for every parameter point, so it is
// computed once per model (in FP64) and the ray kernels skip it.
constexpr int kPlanePrecomputed = 4;

// SIE evaluation in MIXED precision switches to FP64 for every pixel when
// e = sqrt(1 - q^2) < kMixedRoundE, and for the pixels whose square comes
// within kMixedCoreFactor * s / q of the lens centre.
constexpr double kMixedRoundE = 0.05;
constexpr double kMixedCoreFactor = 2.0;

// Series in e replaces atan/atanh below this (both precisions).
constexpr double kSeriesE = 1e-3;

// Sersic b_n table: piecewise Chebyshev series in log n over
// [kBnMin, kBnMax], kBnSeg segments of degree kBnDeg (relative error ~3e-15);
// outside that range the prologue solves for b_n by Newton.
constexpr double kBnMin = 0.2, kBnMax = 12.0;
constexpr int kBnSeg = 32, kBnDeg = 12;

struct SysDev {
    int nx, ny, npix;
    float h, h_lo;       // pixel side as a float pair (h ~ h + h_lo)
    double hd;
    float cx, cy;        // (nx-1)/2, (ny-1)/2
    int nn;              // 1-D nodes of the rule
    int node_off;        // into the 1-D node tables
    int w2_off;          // into the 2-D weight tables (nn * nn)
    int psf_p, psf_q;    // PSF half sizes (0, 0 without a PSF)
    int psf_off;         // into the flipped, normalised PSF table
    long long pix_off;   // into data / weights / per-point image scratch
    int comp_off, ncomp; // into the component tables
    int n_params;
    long long need_off;  // into the needed-pixel list
    int n_need;          // length of the needed-pixel list
    int tile_off, n_tiles;  // into the active-tile list
    int tiles_x, tiles_y;   // full tiling of the image
    double zeropoint;
    int imgpos_mask;        // bit c: component c is a source placed by an image-plane prior
    long long pre_off;      // into the precomputed luminosity table, -1 if none
    int psf_rank;           // > 0: the PSF is applied as a sum of psf_rank separable terms
    int psf_sep_off;        // into the float PSF table: per term, column then row factor
    // the pixel weights are stored relative to this per-system scale (their
    // largest value), which multiplies the chi^2 in FP64 at the end: a
    // uniform weight is then exactly 1 in float, and the float rounding of
    // the weights cannot bias the whole log-likelihood coherently
    double wscale;
};

// Trace-kernel block table entry: system and the range [start, end) of its
// pixel list (or of its pixel indices when the list is the identity).
struct TraceBlock {
    int sys;
    int start, end;
};

// Quadrature nodes: 1-D offsets t*h from the pixel centre, and the 2-D
// weights W_a W_b (float copy adjusted so that it sums to one).
// pre_f / pre_d: per-pixel luminosity of the components that do not depend
// on the parameter point (see kPlanePrecomputed), at SysDev::pre_off; NULL
// while that table is being computed.
struct NodeTables {
    const float *u, *w;
    const double *ud, *wd;
    const float *pre_f;
    const double *pre_d;
    int ff;  // LENSED_PREC_MIXED_FF: re-trace rays near source centres in float-float
};

// PSF-kernel block table entry: system and tile origin.
// An output tile of the PSF kernels.  live_rows: bit r set when output row
// i0 + r carries a weighted pixel; live_warps: bit w set when the 16 x 16
// outputs of warp w (rows 16 (w >> 2) .., columns 16 (w & 3) ..) carry one
// (both all-ones for render tiles).  The mask is fixed per model, so these
// are computed once on the host.
struct PsfBlock {
    int sys;
    int tile;  // global index into the partial-sum columns
    int i0, j0;
    unsigned live_rows, live_warps;
};
static_assert(kTileH == 32 && kTileW == 64 && kPsfThreads == 256,
              "PsfBlock masks: 32 output rows, 8 warps of 16 x 16 outputs");

struct LaunchCfg {
    int trace_threads;  // threads per trace block, one pixel each
    int psf_sep;        // 1: PSFs of low rank run as separable passes
    int ff_split;       // 1 (MIXED_FF): float-float re-traces in a second kernel
    int persistent;     // 1: the trace runs as a persistent, work-queued launch
};

// One deferred float-float ray of a trace launch: lin = the pixel's index in
// the launch's image scratch ((point - p0) * stride + pixel offset of the
// system + pixel), sr = system << 8 | ray index in the rule grid (row-major,
// b * nn + a).  A pixel's entries are consecutive and in ray order.
// lin == kFfNone marks a slot left empty.
struct FfEntry {
    unsigned lin, sr;
};
constexpr unsigned kFfNone = 0xffffffffu;

// MIXED_FF second-pass queues of one trace launch.  cnt[0] = ray entries
// reserved, cnt[1] = pixel records reserved (both zeroed before the launch).
// pix[pcap]: the pixels with a ray near a source centre (FfEntry with
// sr = system), recomputed by k_refine_ff, which puts their rays in
// ent[ecap]; val[ecap] is their source-plane brightness (k_retrace_ff).
// cnt == nullptr: every block re-traces its own rays (no second pass).
struct FfQueue {
    unsigned long long *cnt;
    FfEntry *ent;
    float *val;
    long long ecap;
    FfEntry *pix;
    long long pcap;
    uint2 *prun;  // [pcap]: each pixel record's rays in ent (first, count; count 0: none queued)
};

// True when the test hook lensed_debug_fail_alloc says the next device
// allocation must fail (every allocator of the library asks before
// cudaMalloc).  Defined in lensed_runtime.cu.
bool alloc_failure_injected();
// Count of live device buffers of the library (+1 per allocation, -1 per
// free), reported by lensed_debug_fail_alloc.
void note_buffers(int delta);

// --- kernels launched from the runtime (defined in lensed_kernels.cu) ---

// a1: per (system, point) packed constants and validity.
// a1 for components c0 .. c0+nC-1 (global indices, belonging to systems
// s0 .. s0+nS-1) and points p0 .. p0+nP-1; with single_row, params is one
// row (the render path).  cvalid: [P][C_total] scratch bytes.
void launch_prologue(const SysDev *sys, const int *comp_sys, int s0, int nS, int c0, int nC,
                     const int *comp_type, const int *comp_free, const double *comp_value,
                     const double *params, bool single_row, int P, int p0, int nP,
                     int n_par_stride, int C_total, const double *bn_table, float *cf,
                     double *cd, unsigned char *cvalid, unsigned char *valid, cudaStream_t st);

// a2-a5: pixel luminosities of the pixels in the block table, for points
// p0 .. p0 + nP - 1, into Lbuf[(p - p0) * L_stride + pix_off + pix].  Every
// system in the table has nn nodes per row of its rule.  MIXED_FF with
// cfg.ff_split and a queue (q.cnt != nullptr): the float-float re-traces run
// in a second kernel after the first (same results bit for bit).
void launch_trace(int precision, LaunchCfg cfg, int nn, const SysDev *sys, const int *comp_type,
                  const int *comp_plane, const float *cf, const double *cd,
                  const unsigned char *valid, int P, int C_total, const TraceBlock *blocks,
                  int n_blocks, const int *need, NodeTables nodes, int p0, int nP, void *Lbuf,
                  long long L_stride, cudaStream_t st, FfQueue q = FfQueue{},
                  unsigned long long *work = nullptr);

// One-time kernel attributes (dynamic shared memory limits); call before
// any launch or capture.
void init_kernel_attributes();

// MIXED only: recompute, with the FP64 SIE, the pixels of each (system,
// point) that the MIXED rule assigns to FP64 (after launch_trace wrote
// their FP32 values).  need == nullptr: every pixel of the systems (render).
void launch_fix64(LaunchCfg cfg, const SysDev *sys, int s0, int nS, const int *comp_type,
                  const int *comp_plane, const float *cf, const double *cd,
                  const unsigned char *valid, int P, int C_total, const int *need,
                  NodeTables nodes, int p0, int nP, void *Lbuf, long long L_stride,
                  cudaStream_t st);

// a6-a7: PSF convolution of the tiles in the block table, then either the
// masked chi^2 partial sums (partial != nullptr) or the convolved image
// (out != nullptr, one point).  sep > 0 (FP32 modes): every system of the
// table applies its PSF as SysDev::psf_rank <= sep separable terms.
void launch_psf(int precision, int q, int sep, int p_max, const SysDev *sys, const float *psf_f,
                const double *psf_d, const float *data, const float *weight,
                const double *data_d, const double *weight_d,
                const unsigned char *valid, int P, const PsfBlock *blocks, int n_blocks, int p0,
                int nP, const void *Lbuf, long long L_stride, double *partial, int T_total,
                float *out, cudaStream_t st);

// a7: loglike = -1/2 sum of the partials of each (system, point).
void launch_finalize(const SysDev *sys, const unsigned char *valid, int P,
                     const double *partial, int T_total, double *out, int s0, int p0, int nS,
                     int nP, cudaStream_t st);

// Copy an unconvolved image out of the scratch buffer (render path).
void launch_copy_image(int precision, const void *Lbuf, long long off, int npix,
                       const unsigned char *valid, float *out, cudaStream_t st);

// Throughput probes (FMA or MUFU ex2 chains) for the measured ALU peaks.
void launch_probe(int mufu, int blocks, int threads, int iters, float *sink, cudaStream_t st);
void launch_trig_probe(const float *n, const float *d, long long count, float *out,
                       cudaStream_t st);

// |L_K - L_G| of one system's pixels (the Gauss-Kronrod error estimate),
// NaN if the point is invalid.
void launch_error_image(int precision, const void *LK, const void *LG, long long off, int npix,
                        const unsigned char *valid, float *out, cudaStream_t st);

}  // namespace lensed
