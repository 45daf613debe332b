// The handle behind the opaque sbec_handle of the C ABI (shared by the C-ABI
// and solver translation units).
#pragma once

#include <cuda_runtime.h>

#include "sbec.h"
#include "sbec_internal.h"

struct sbec_handle {
    sbec_problem prob;
    sbec::Geom geom;
    sbec::Work work;
    cudaStream_t stream;
    int device;
    size_t elem;          // bytes of one complex value
    size_t field_bytes;   // C * G * elem
    void* d_tw;
    double* d_lam2;
    void* d_V;
    void* stage[3];
    const void* stage0_src;   // host array whose contents stage[0] received last (null: none known)
    double* h_scal;       // pinned mirror of the scalar block
    const void* last_grad_X;
    sbec::Prof prof;
    int B;                // instances of a batch handle (1 for sbec_create)
    void* d_ppb;          // per-instance PointParams (batch handles)
    double* d_Mb;         // per-instance magnetisations (batch handles)
    int* d_imap;          // launch slot -> instance map of a batch solve (B ints, device)
    int* h_imap;          // its pinned host mirror
};

// helpers of the C-ABI translation unit used by the solver
int sbec_read_scalars(sbec_handle* h);
bool sbec_is_device_ptr(const void* p);
