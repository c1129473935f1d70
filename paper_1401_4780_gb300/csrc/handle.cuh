// handle.cuh -- host-side state behind an asyrk_problem handle (device
// pointers, sizes, lazily allocated workspace).  No kernel reads this struct:
// kernels get their arguments by value (ProjArgs and the launch parameters).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

struct RowRec;

struct asyrk_problem {
    int64_t m = 0, n = 0, nnz = 0, nnz_pad = 0, max_len = 0;
    int dtype = 0;
    int uniform = 0;
    int device = 0;
    int sm_count = 0;
    uint64_t seed = 0;
    uint64_t j_next = 0;
    double frob2 = 0.0;
    double bnorm = 0.0;
    int64_t dev_bytes = 0;
    bool rec_b_is_residual = false;  // rec[i].b currently holds a refinement residual
    int64_t launches = 0;            // kernels launched on behalf of this handle
    int64_t lsq_n = 0;               // > 0: the least-squares system of an m x lsq_n matrix
    double lsq_zeta = 0.0;           //      its y-block scale zeta (as stored)
    double lsq_phi = 0.0;            //      and its A^T-block scale phi

    RowRec *rec = nullptr;
    int32_t *col = nullptr;
    void *val = nullptr;
    double *b64 = nullptr;
    double *w64 = nullptr;

    // solve workspace, allocated on first use
    void *xw = nullptr;          // n x {float|double}: the shared iterate
    double *x64 = nullptr;       // n: FP64 iterate / staging
    double *xt64 = nullptr;      // n: x*
    double *g64 = nullptr;       // n: A^T (A x - b) (Table 2's measure), allocated on use
    double *red_part = nullptr;  // reduction partials
    unsigned *red_count = nullptr;
    double *red_out = nullptr;   // 8 result slots
    double *h_out = nullptr;     // pinned host copy of red_out
    unsigned *busy = nullptr;              // ceil(m/32) row-claim words, zero between launches
    unsigned long long *skipped = nullptr; // projections skipped by row exclusion
    int32_t *rows_buf = nullptr;
    int64_t rows_cap = 0;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    void *loop_state = nullptr;        // device state of the graph-captured solve loop
    cudaStream_t cap_stream = nullptr; // stream the loop body is captured on
};
