// group.cuh -- internal: the grouped plan (plv_group) and the host-side
// layouts of its two work lists, shared by the plan builder (plv_api.cu) and
// the autotuner (tune.cu).  Not part of the public ABI.
#pragma once

#include <map>
#include <string>
#include <vector>

#include "common.cuh"

namespace plv {

// Makes a device current for the scope and restores the caller's.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev)
            cudaSetDevice(prev);
    }
};

}  // namespace plv

struct plv_group {
    int device = 0;
    plv_precision prec = PLV_PREC_FP32;
    std::vector<plv_problem> host;   // validated problems (FP32 path)
    unsigned mask = 0;
    plv::TcProblem *probs = nullptr;  // device descriptors (split paths)
    int4 *items = nullptr;            // device tile list
    int nprob = 0, nitems = 0;
    bool any_diag = false;
    std::vector<plv::TcProblem> dp_host;  // host copies of the descriptors
    std::vector<int4> items_host;         // tile list, longest first
    // analytic-signal plan (problems with an input x)
    bool has_k1 = false;
    plv_dtype k1_dtype = PLV_F32;
    plv::K1Desc *k1_descs = nullptr;  // device
    int2 *k1_items = nullptr;         // device
    plv::K1Group k1{};
    std::vector<plv::K1Desc> k1_host;  // host copies of the K1 descriptors
    plv::GroupConfig cfg;              // current launch configuration
    // work lists replaced by the autotuner, kept until the plan is destroyed
    // (CUDA graphs captured before tuning still launch on them)
    std::vector<void *> retired;
};

namespace plv {

// The (problem, row pair) items of a grouped K1 plan: by assigned thread
// class (cls[M], default conv_class(M)), then by decreasing M, then problem
// order.  Fills kg's begin / count / max_M (per_sm, descs and items are left
// to the caller).
void k1_layout(const std::vector<K1Desc> &descs, const std::map<int, int> &cls,
               std::vector<int2> &items, K1Group &kg);

// The grouped Gram's tile list in the given schedule, from the longest-first
// list `sorted` (stable by decreasing K blocks); G is the persistent grid.
std::vector<int4> gram_order(const std::vector<TcProblem> &dp, const std::vector<int4> &sorted,
                             int schedule, int G, int tile_cost);

// The persistent grid of the grouped Gram launch for n tiles.
inline int gram_group_grid(const Handle &h, int n) { return n < h.num_sms ? n : h.num_sms; }

}  // namespace plv
