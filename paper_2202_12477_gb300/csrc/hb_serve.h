// Internal declarations of the CG server: the per-slot descriptor and solve
// state that the serving kernels read from device memory.
#pragma once

#include "hb_internal.h"

#define HB_SERVE_MAX_N 11     // degrees the server accepts
#define HB_SERVE_GRID 304     // fixed grid of the serving vector kernels (2 x 152 SMs)
#define HB_SERVE_AXP 1024     // room for the FP32 element kernels' block partials (their grids are smaller)
#define HB_SERVE_THREADS 256

enum { HB_SLOT_EMPTY = 0, HB_SLOT_OUTER = 1, HB_SLOT_INNER = 2, HB_SLOT_DONE = 3 };

// Everything a slot's kernels need, in device memory (one per slot position).
struct hb_slot_desc {
    int active;
    int N;
    int screen;
    int max_it, max_outer;
    int pad0;
    int64_t E, n_local, n_global, nsr;
    const int32_t *l2g, *srow_g, *srowptr, *scols;
    const double *geo;
    const float *geo32;
    const double *mdiag;
    const float *mdiag32;
    void *ysurf;                  // surface store (n_local doubles of room)
    const double *b;
    double *x, *r, *Ap;           // FP64 solution, residual, A x
    float *r32, *p32, *Ap32, *d32;  // FP32 inner CG
    double lambda, rtol, inner_rtol;
    double *partials;             // [HB_RED_MAXV * HB_RED_BLOCKS]
    double *ax_partials;          // [HB_SERVE_AXP], zero past the element kernel's grid
    unsigned *counters;           // [8]
};

// Solve state of a slot (FP32-inner / FP64 defect-correction CG).
struct hb_slot_state {
    hb_cg_state outer;  // FP64 residual: rr, bb
    hb_cg_state inner;  // FP32 inner CG
    int phase;          // HB_SLOT_*
    int x_pending;      // 1 when x += ||r|| d32 is due
    int outer_it;
    int inner_total;
    int status;
    int pad[3];
};

// Element kernels of the server (one per precision translation unit):
// FP64: A x of the slot's current solution into Ap (runs when phase == OUTER);
// FP32: A p32 into Ap32 with the interior partials of p.Ap (runs while the
// inner CG runs).
hb_status hb_serve_launch_ax_f64(const hb_slot_desc *d, const hb_slot_state *st, cudaStream_t s);
hb_status hb_serve_launch_ax_f32(const hb_slot_desc *d, const hb_slot_state *st, cudaStream_t s);
size_t hb_serve_ax_smem_f64();
size_t hb_serve_ax_smem_f32();
