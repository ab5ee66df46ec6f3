// Autotuning of launch schedules: the lanes-per-surfel mapping of a plan and the (mapping variant,
// surfels per work item) schedule of a batch are chosen by timing the real solve on the bound stream
// with CUDA events.  Results can be kept in a plain-text cache file, one "key value..." line per
// tuned configuration, keyed by the GPU name and the shape of the problem.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "sgn.h"
#include "sgn_internal.h"

extern "C" sgn_status sgn_plan_desc_default(sgn_plan_desc*, int, int, int, int);

namespace {

sgn_status tune_error(sgn_status st, const std::string& msg) { return sgn::record_error(st, msg.c_str()); }

std::string gpu_name() {
    int dev = 0;
    cudaDeviceProp prop{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    std::string n = prop.name;
    for (char& c : n)
        if (c == ' ' || c == '|') c = '_';
    return n;
}

bool cache_lookup(const char* path, const std::string& key, std::vector<int>* values) {
    if (!path || !*path) return false;
    std::ifstream in(path);
    std::string line;
    bool found = false;
    while (std::getline(in, line)) {  // the last matching line wins
        std::istringstream ls(line);
        std::string k;
        if (!(ls >> k) || k != key) continue;
        std::vector<int> v;
        int x;
        while (ls >> x) v.push_back(x);
        *values = v;
        found = true;
    }
    return found;
}

void cache_store(const char* path, const std::string& key, const std::vector<int>& values) {
    if (!path || !*path) return;
    std::ofstream out(path, std::ios::app);
    out << key;
    for (int v : values) out << ' ' << v;
    out << '\n';
}

// Median time (ms) of `reps` runs of fn on `stream`, after one warm-up run.
template <class Fn>
sgn_status time_median(cudaStream_t stream, int reps, Fn fn, float* ms) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
        return tune_error(SGN_ERR_CUDA, "autotune: cudaEventCreate failed");
    std::vector<float> t;
    sgn_status st = fn();
    for (int r = 0; r < reps && st == SGN_OK; ++r) {
        cudaEventRecord(a, stream);
        st = fn();
        cudaEventRecord(b, stream);
        if (st != SGN_OK) break;
        if (cudaEventSynchronize(b) != cudaSuccess) {
            st = tune_error(SGN_ERR_CUDA, "autotune: kernel failed while timing");
            break;
        }
        float x = 0.0f;
        cudaEventElapsedTime(&x, a, b);
        t.push_back(x);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != SGN_OK) return st;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return SGN_OK;
}

}  // namespace

// Plan internals needed here (kept in api.cpp).
extern "C" sgn_status sgn_plan_set_mapping(sgn_plan*, int, int);
namespace sgn {
cudaStream_t plan_stream(const sgn_plan* p);
void plan_shape(const sgn_plan* p, int* W, int* H, int* P, int* F, int* dtype);
cudaStream_t batch_stream(const sgn_batch* b);
std::string batch_signature(const sgn_batch* b);
}  // namespace sgn

extern "C" sgn_status sgn_plan_autotune(sgn_plan* plan, int iters, const char* cache_path, int* lanes_out,
                                        int* block_out) {
    if (!plan) return tune_error(SGN_ERR_INVALID_ARGUMENT, "plan is NULL");
    int W, H, P, F, dt;
    sgn::plan_shape(plan, &W, &H, &P, &F, &dt);
    std::ostringstream key;
    key << "plan|" << gpu_name() << '|' << W << 'x' << H << "|P" << P << "|F" << F << "|dt" << dt << "|it" << iters;
    std::vector<int> v;
    if (cache_lookup(cache_path, key.str(), &v) && v.size() == 2 && sgn_plan_set_mapping(plan, v[0], v[1]) == SGN_OK) {
        if (lanes_out) *lanes_out = v[0];
        if (block_out) *block_out = v[1];
        return SGN_OK;
    }
    std::vector<int> lanes = P == 4 ? std::vector<int>{8, 16} : (P == 8 ? std::vector<int>{8, 16, 32} : std::vector<int>{32});
    const int blocks[] = {128, 256};
    float best = 1e30f;
    int bl = 0, bb = 0;
    for (int G : lanes)
        for (int B : blocks) {
            sgn_status st = sgn_plan_set_mapping(plan, G, B);
            if (st != SGN_OK) return st;
            float ms = 0.0f;
            st = time_median(sgn::plan_stream(plan), 3, [&] { return sgn_solve(plan, iters); }, &ms);
            if (st != SGN_OK) return st;
            if (ms < best) {
                best = ms;
                bl = G;
                bb = B;
            }
        }
    sgn_status st = sgn_plan_set_mapping(plan, bl, bb);
    if (st != SGN_OK) return st;
    cache_store(cache_path, key.str(), {bl, bb});
    if (lanes_out) *lanes_out = bl;
    if (block_out) *block_out = bb;
    return SGN_OK;
}

extern "C" sgn_status sgn_batch_autotune(sgn_batch* batch, int iters, const char* cache_path, int* variant_out,
                                         int* chunk_out) {
    if (!batch) return tune_error(SGN_ERR_INVALID_ARGUMENT, "batch is NULL");
    const std::string key = "batch|" + gpu_name() + '|' + sgn::batch_signature(batch) + "|it" + std::to_string(iters);
    std::vector<int> v;
    if (cache_lookup(cache_path, key, &v) && v.size() == 2 && sgn_batch_set_schedule(batch, v[0], v[1]) == SGN_OK) {
        if (variant_out) *variant_out = v[0];
        if (chunk_out) *chunk_out = v[1];
        return SGN_OK;
    }
    const int chunks[] = {8, 16, 32, 64, 128, 256};
    float best = 1e30f;
    int bv = 0, bc = 64;
    for (int var = 0; var < 3; ++var)
        for (int ch : chunks) {
            if (var == 2 && ch != chunks[0]) continue;  // square items: the chunk only applies to other kinds
            sgn_status st = sgn_batch_set_schedule(batch, var, ch);
            if (st != SGN_OK) return st;
            size_t need = 0;
            sgn_batch_workspace_bytes(batch, &need);
            float ms = 0.0f;
            st = time_median(sgn::batch_stream(batch), 3, [&] { return sgn_batch_run(batch, iters); }, &ms);
            if (st == SGN_ERR_WORKSPACE_TOO_SMALL) continue;  // smaller chunks need a longer work list
            if (st != SGN_OK) return st;
            if (ms < best) {
                best = ms;
                bv = var;
                bc = ch;
            }
        }
    if (best >= 1e30f) return tune_error(SGN_ERR_WORKSPACE_TOO_SMALL, "autotune: no schedule fits the batch workspace");
    sgn_status st = sgn_batch_set_schedule(batch, bv, bc);
    if (st != SGN_OK) return st;
    cache_store(cache_path, key, {bv, bc});
    if (variant_out) *variant_out = bv;
    if (chunk_out) *chunk_out = bc;
    return SGN_OK;
}
