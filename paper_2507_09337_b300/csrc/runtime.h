// runtime.h -- host-side runtime objects behind the opaque C-ABI handles
// (internal to the library).
#pragma once

#include <vector>

#include "../../include/orcha.h"
#include "common.cuh"
#include "persistent.cuh"
#include "launch.h"

namespace orcha {

// A captured multi-step sequence of one mesh (orcha_mesh_advance).
struct GraphEntry {
    std::vector<const orcha_packet*> packets;
    orcha_task task;
    int nsteps, init_dt, start_cur;
    cudaGraphExec_t exec;
};

}  // namespace orcha

struct orcha_mesh {
    orcha_mesh_desc desc;
    orcha::MeshDev dev;
    int cur = 0;
    int nblk = 0;
    long long ncell = 0;             // interior cells per block
    unsigned long long* smax = nullptr;
    int* err = nullptr;
    double* staging = nullptr;       // device staging of interior arrays for host load/store
    int tile_x = 8, tile_y = 8;
    int device = 0;
    std::vector<orcha::GraphEntry> graphs;
};

struct orcha_packet {
    orcha_mesh* mesh;
    int n;
    int* ids_dev;
    std::vector<int> ids;
    double* staging = nullptr;       // device staging of the packet's interiors for host pack/unpack
};

struct orcha_batch {
    std::vector<orcha_mesh*> meshes;                 // one slot per mesh
    std::vector<const orcha_packet*> packets;
    int ndim = 3, tx = 8, ty = 8;
    std::vector<orcha::Item> base_items;             // full-block items in packet order
    // per precision (orcha::Prec): work list sized for that variant's occupancy
    struct List {
        bool built = false;
        int nitems = 0, grid = 0;
        orcha::Item* items_dev = nullptr;
        orcha::SlotDev* slots_dev = nullptr;
        unsigned* done_dev = nullptr;
        double* scratch = nullptr;                   // fused variants: per-CTA intermediate state
        long long per_cta = 0;                       // its doubles per CTA
        unsigned long long* smax2 = nullptr;         // two-step variants: intermediate state's block speeds
        unsigned long long* sub = nullptr;           // one-step variants: skipped cells' speed bounds per block
    } lists[orcha::kNumPrec];                        // indexed by orcha::Prec
    unsigned* queue = nullptr;
    int* cur_dev = nullptr;
    int num_sms = 0;
    struct G { orcha_task task; int nsteps; cudaGraphExec_t exec; };
    std::vector<G> graphs;
};
