// Persistent interleaved work queue (ef_queue.cu): declarations shared by the
// single-mesh path (ef_api.cu) and the batch (ef_batch.cu).
#pragma once

#include <vector>

#include "ef_internal.cuh"

namespace ef {

struct QueueMesh {              // device-side view of one mesh's plan
    const int32_t* elems;
    const uint32_t* inv;        // element contribution -> work-ordered list position
    const uint32_t* wseg;       // work item -> list range
    const uint32_t* wpos_up;    // work item -> CSR position of (r,c)
    const uint32_t* wpos_lo;    // work item -> CSR position of (c,r) or 0xffffffff
    const void* wst_up;         // store orders of the sum kernel (ef_assemble.cu)
    const void* wst_lo;
    double2* list;              // np * T contribution values, (K, M) pairs
    const double* nodes;        // bound buffers (batch); the single-mesh path passes them per call
    const double* coeff;
    double* K;
    double* M;
    int64_t T, U;
};

struct QueueSegment {           // a run of tiles of one kind for one (mesh, chunk)
    int32_t type;               // 0: element tiles, 1: sum tiles
    int32_t mesh;
    int32_t chunk;              // element chunk index x (element segments: the counter it bumps)
    int32_t dep_first;          // sum segments: element chunks dep_first .. dep_first+dep_count-1 must be done
    int32_t dep_count;
    int32_t pad;
    int64_t lo, hi;             // element range (type 0) or work-item range (type 1)
    int64_t ntiles;
    int64_t tile_off;           // first tile of this segment in queue order
};

struct QueueArgs {              // per-call buffers of the single-mesh path (all NULL for a batch)
    const double* nodes = nullptr;
    const double* coeff = nullptr;
    double* K = nullptr;
    double* M = nullptr;
};

struct Queue {
    int variant = 0;
    int sms = 0;
    ef_batch_config_t cfg{};
    std::vector<QueueMesh> host_mesh;
    QueueMesh* d_mesh = nullptr;
    QueueSegment* d_seg = nullptr;
    uint32_t* d_need = nullptr;   // element tiles of each element chunk
    uint32_t* d_ctrl = nullptr;   // [0] ticket, [1] exited, [2] sum ticket, [3 + x] done tiles of element chunk x
    int* d_status = nullptr;
    bool own_status = true;
    int nseg = 0, nctr = 0;
    int64_t ntiles = 0;
    int64_t n_elem_tiles = 0;     // role split: tiles [0, n_elem_tiles) are element tiles
    int cap_mesh = 0, cap_seg = 0, cap_ctr = 0;
    // two-launch schedule: first element block / first sum block of each
    // mesh, and the mesh of every element block / sum block
    int64_t* d_eblk = nullptr;
    int64_t* d_sblk = nullptr;
    uint32_t* d_emesh = nullptr;
    uint32_t* d_smesh = nullptr;
    int64_t n_eblk = 0, n_sblk = 0;
    int64_t cap_eblk = 0, cap_sblk = 0;
    int nmesh = 0;
    uint32_t stall = 0;           // fault injection: extra tiles the first element chunk must report
};

int queue_init(Queue* q, int variant, int* shared_status);
void queue_free(Queue* q);
int queue_set_meshes(Queue* q, const std::vector<ef_plan*>& plans, cudaStream_t s);
int queue_build(Queue* q, const std::vector<ef_plan*>& plans, cudaStream_t s);
int queue_launch(const Queue* q, const QueueArgs& a, cudaStream_t s);
int queue_check(const Queue* q, cudaStream_t s);
int queue_inject_stall(Queue* q, int on, cudaStream_t s);
int queue_max_ctas_per_sm(int variant, int BE);

// Batch in two launches (ef_assemble.cu): the element kernel over every
// mesh's elements, then the sum kernel over every mesh's work items.
int launch_batch_two_pass(int variant, const QueueMesh* d_mesh, const uint32_t* d_emesh, const int64_t* d_eblk,
                          int64_t n_eblk, const uint32_t* d_smesh, const int64_t* d_sblk, int64_t n_sblk, int* status,
                          cudaStream_t s);
int64_t element_blocks(int64_t T);
int64_t sum_blocks(int64_t U);

}  // namespace ef
