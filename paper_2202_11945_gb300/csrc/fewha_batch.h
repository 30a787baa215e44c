// Batched frames of many independent FEWHA instances (uneven sizes): the per-frame
// sequence of Algorithm 1 is the same list of steps for every instance, so step j of all
// instances runs as ONE launch over a work list of (instance, unit) items, where a unit
// is a layer, a sensor, a (sensor, layer) pair or a CTA of the vector / fit kernels.
// Each CTA reads its instance's descriptor and its step arguments from device arrays.
#pragma once

#include <cuda_runtime.h>

#include "fewha_pair.cuh"

namespace fewha {

// One work item: instance index and unit within the instance (a pair is g * MAXL + l).
struct BItem {
    int inst;
    int unit;
};

// Per-instance constant data of a batched launch, in device memory.
template <class T>
struct alignas(16) BInst {
    Desc<T> d;
    ClLayout lay_fwd, lay_inv;
    SensorLayout lay_sen;
    PairBufs<T> pb;
    int desc_bytes;     // leading bytes of d that the kernels read (through the last sensor's boxes)
    unsigned ctas_layer;  // CTAs of the instance in a layer-cluster launch (CL * n_layers)
    int nparts;         // CTAs of the instance in a vector launch
};

// Arguments of the DM fit step.
template <class T>
struct FitArgs {
    const T* phi;
    T* a_prev;
    T* out;
    int apply_gain;
    const T* cpist;     // c, when phi lacks the full layers' pistons (carried layers)
};

// Step kinds of the frame (each names one kernel template instance).
enum BKind {
    BK_INV = 0,        // phi = W^T c                       (ClArgs)
    BK_INV_UPD,        // p = z + beta p, phi = W^T p       (ClArgs)
    BK_PROJ,           // pair terms of P phi               (const T*: phi)
    BK_SEN_PHI,        // Gamma, C^-1, Gamma^T of P phi     (SensorArgs)
    BK_SEN_SLOPES,     // C^-1, Gamma^T of measured slopes  (SensorArgs)
    BK_PROJT,          // pair terms of P^T u               (const T*: u)
    BK_FWD_APPLY,      // q = W sum P^T u + alpha D p, p.q  (ClArgs)
    BK_FWD_COEF,       // b = W sum P^T u                   (ClArgs)
    BK_VEC_INIT,       // r0 = b - q, z, p, r.z             (VecArgs)
    BK_VEC_WARM,       // r0 = (b - b_prev) + r_prev        (VecArgs)
    BK_VEC_UPDATE,     // CG update                         (VecArgs)
    BK_FIT,            // DM fit and gain                   (FitArgs)
    BK_SEN_RESID,      // C^-1, Gamma^T of s - Gamma P phi  (SensorArgs)
    BK_FWD_RINIT,      // r0 = W sum P^T u - alpha D c0, z0, p0, r.z (ClArgs)
    BK_COUNT
};

// Which work list a step kind runs over.
enum BList { BL_LAYER = 0, BL_SENSOR, BL_PAIR, BL_VEC, BL_FIT, BL_COUNT };

inline int bkind_list(int kind) {
    switch (kind) {
        case BK_INV: case BK_INV_UPD: case BK_FWD_APPLY: case BK_FWD_COEF: case BK_FWD_RINIT: return BL_LAYER;
        case BK_SEN_PHI: case BK_SEN_SLOPES: case BK_SEN_RESID: return BL_SENSOR;
        case BK_PROJ: case BK_PROJT: return BL_PAIR;
        case BK_FIT: return BL_FIT;
        default: return BL_VEC;
    }
}

// One batched launch.
struct BLaunch {
    int kind;
    const void* inst;      // BInst<T>[count]
    const void* args;      // per-instance arguments of this step (type by kind)
    const BItem* items;    // work list
    int n_items;
    size_t smem;           // dynamic shared memory (max over the instances present)
    bool pdl;              // programmatic stream serialization (see FEWHA_FLAG_PDL)
    int pair_nt;           // threads of the projection kernels: cblk<T>() or half of it
    int taps;              // unrolled taps of the adjoint projection: 4 or KMAX
    int vec_nt;            // threads of the vector kernel: PBLK or 2 PBLK
};

// Launch one batched step (defined in fewha_batch.cu for float and double).
template <class T>
cudaError_t batch_launch(const BLaunch& L, cudaStream_t st);

// The db3 taps of the batched kernels: __constant__ memory is per translation unit, so
// this unit's copy is filled separately (per device, before the first batched launch).
cudaError_t batch_set_taps(const double* h, const double* g);

// Largest dynamic shared memory a batched kernel of this kind accepts (over its launch
// shapes); sets the kernels' attribute to it on first use (per device).
template <class T>
cudaError_t batch_smem_limit(int kind, size_t* bytes);

}  // namespace fewha
