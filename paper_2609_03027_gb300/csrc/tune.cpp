// Autotuner of a plan's internal tiling (epic_plan_tune): coordinate descent
// over the path's tuning parameters, each candidate timed with CUDA events on
// the caller's stream over `reps` calls of the caller's block.
#include <algorithm>
#include <string>
#include <vector>

#include "epic_internal.h"

namespace {

struct Knob {
    const char* name;
    std::vector<int> values;
    int current;
    epic_status (*set)(epic_plan_s*, int);
};

epic_status set_plain_chunk(epic_plan_s* p, int mb) { return epic::plain_set_chunk(p, (size_t)mb << 20); }
epic_status set_plain_fft(epic_plan_s* p, int v) { return epic::plain_set_fft(p, v); }
epic_status set_dft_chunk(epic_plan_s* p, int mb) { return epic::dftgemm_set_chunk(p, (size_t)mb << 20); }
epic_status set_dft_frames(epic_plan_s* p, int f) { return epic::dftgemm_grid_config(p, f); }
epic_status set_fused_slab(epic_plan_s* p, int sw) { return epic::fused_set_slab(p, sw); }
epic_status set_dft_kernel(epic_plan_s* p, int v) { return epic::dftgemm_set_kernel(p, v); }
epic_status set_dft_grid_kernel(epic_plan_s* p, int v) { return epic::dftgemm_set_grid_kernel(p, v); }
epic_status set_dft_split(epic_plan_s* p, int v) { return epic::dftgemm_set_split(p, v); }
epic_status set_dft_group(epic_plan_s* p, int v) { return epic::dftgemm_set_group(p, v); }
epic_status set_path(epic_plan_s* p, int v) { return epic::set_path(p, v); }

// the tuning parameters of a plan's path with their candidate and current values
std::vector<Knob> knobs_for(const epic_plan_s* p)
{
    std::vector<Knob> knobs;
    const int budget_mb = (int)(p->chunk_budget >> 20);
    if (p->auto_path)  // EPIC_PATH_AUTO: the path itself, timed first (each path's own knobs follow)
        knobs.push_back({"path", {EPIC_PATH_PLAIN_FP32, EPIC_PATH_FUSED_FP32, EPIC_PATH_DFTGEMM_FP16}, p->path,
                         set_path});
    if (p->path == EPIC_PATH_PLAIN_FP32) {
        knobs.push_back({"fft", {0, 1}, p->plain_fft, set_plain_fft});
        knobs.push_back({"chunk_mb", {128, 256, 512, 1024}, budget_mb, set_plain_chunk});
    } else if (p->path == EPIC_PATH_FUSED_FP32) {
        knobs.push_back({"slab", {8, 16, 32}, p->slab, set_fused_slab});
    } else if (p->path == EPIC_PATH_DFTGEMM_FP16) {
        if (p->tc.ws) knobs.push_back({"group", {0, 1}, p->tc.group, set_dft_group});
        if (p->tc.ws && p->sub == 0) {  // sub-integrations use the control-warp kernel on whole items
            knobs.push_back({"mma_kernel", {1, 2, 3}, p->tc.ws_variant, set_dft_kernel});
            knobs.push_back({"split", {-1, 0, 1}, p->tc.split, set_dft_split});
        }
        if ((p->tc.grid_ps ? 1 : 0) + (p->tc.gtask ? 1 : 0) + (p->tc.pl_ptr ? 1 : 0) >= 2)
            knobs.push_back({"grid_kernel", {1, 2, 3}, p->tc.grid_variant, set_dft_grid_kernel});
        if (p->tc.grid_ps || p->tc.gtask || p->tc.pl_ptr)
            knobs.push_back({"grid_frames", {1, 2, 4, 8}, p->tc.grid_frames, set_dft_frames});
        knobs.push_back({"chunk_mb", {96, 192, 384, 768, 1536, 3072, 6144, 12288, 24576}, budget_mb, set_dft_chunk});
    }
    return knobs;
}

// a recorded graph refers to the previous scratch and launch shapes
void drop_graph(epic_plan_s* p)
{
    if (p->gexec) {
        cudaGraphExecDestroy(p->gexec);
        p->gexec = nullptr;
        p->g_T = -1;
    }
}

// mean ms of one call over reps calls (after one untimed call); negative on error
epic_status time_calls(epic_plan_s* p, const uint8_t* volt, int T, cudaStream_t s, float* out, int reps,
                       cudaEvent_t e0, cudaEvent_t e1, float* ms)
{
    epic_status st = epic::image_run(p, volt, T, s, out, EPIC_RESET);
    if (st != EPIC_OK) return st;
    cudaError_t e = cudaEventRecord(e0, s);
    for (int r = 0; r < reps && st == EPIC_OK; ++r) st = epic::image_run(p, volt, T, s, out, EPIC_RESET);
    if (st != EPIC_OK) return st;
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e != cudaSuccess) return epic::cuda_fail(p, e, "autotuner timing");
    *ms = t / reps;
    return EPIC_OK;
}

}  // namespace

extern "C" epic_status epic_plan_tune(epic_plan_t p, const uint8_t* volt, int T, void* stream, float* out, int reps,
                                      epic_tune_report* rep)
{
    if (!p) return EPIC_ERR_INVALID_ARG;
    if (!volt || !out || T < 1 || T > p->max_time || reps < 1 || reps > 100) {
        p->last_error = "tune: need device volt and out, 1 <= T <= max_time, 1 <= reps <= 100";
        return EPIC_ERR_INVALID_ARG;
    }
    cudaPointerAttributes at{};
    auto on_device = [&](const void* ptr) {
        return cudaPointerGetAttributes(&at, ptr) == cudaSuccess &&
               (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    };
    if (!on_device(volt) || !on_device(out)) {
        cudaGetLastError();
        p->last_error = "tune: voltage and image pointers must be device memory";
        return EPIC_ERR_INVALID_ARG;
    }
    const cudaStream_t s = (cudaStream_t)stream;
    p->timing = false;

    drop_graph(p);
    std::vector<Knob> knobs = knobs_for(p);
    const bool path_knob = p->auto_path;

    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return epic::cuda_fail(p, e, "cudaEventCreate(tune)");
    }
    int timed = 0;
    float base_ms = 0.f, best_ms = 0.f;
    epic_status st = time_calls(p, volt, T, s, out, reps, e0, e1, &base_ms);
    best_ms = base_ms;
    ++timed;
    for (size_t k = 0; k < knobs.size() && st == EPIC_OK; ++k) {
        Knob& kb = knobs[k];
        int best_v = kb.current;
        for (int v : kb.values) {
            if (v == kb.current) continue;
            epic_status sv = kb.set(p, v);
            if (sv == EPIC_ERR_UNSUPPORTED) continue;
            if (sv != EPIC_OK) {
                st = sv;
                break;
            }
            float ms = 0.f;
            st = time_calls(p, volt, T, s, out, reps, e0, e1, &ms);
            if (st != EPIC_OK) break;
            ++timed;
            if (ms < best_ms) {
                best_ms = ms;
                best_v = v;
            }
        }
        // leave the knob at its best value (the previous one when nothing beat it)
        epic_status sb = kb.set(p, best_v);
        if (st == EPIC_OK) st = sb;
        kb.current = best_v;
        if (path_knob && k == 0) {  // the path is chosen: tune its own parameters next
            std::vector<Knob> rest = knobs_for(p);
            knobs.resize(1);
            knobs.insert(knobs.end(), rest.begin() + 1, rest.end());
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rep) {
        rep->n_timed = timed;
        rep->default_ms = base_ms;
        rep->best_ms = best_ms;
        rep->n_params = (int)std::min<size_t>(knobs.size(), 8);
        for (int i = 0; i < rep->n_params; ++i) {
            rep->names[i] = knobs[i].name;
            rep->values[i] = knobs[i].current;
        }
    }
    return st;
}

extern "C" epic_status epic_plan_set_param(epic_plan_t p, const char* name, int value)
{
    if (!p || !name) return EPIC_ERR_INVALID_ARG;
    for (Knob& kb : knobs_for(p)) {
        if (std::string(kb.name) != name) continue;
        drop_graph(p);
        epic_status st = kb.set(p, value);
        if (st == EPIC_ERR_UNSUPPORTED) p->last_error = std::string("value not possible for parameter ") + name;
        else if (st == EPIC_OK) cudaGetLastError();
        return st;
    }
    p->last_error = std::string("no tuning parameter named ") + name + " on this plan's path";
    return EPIC_ERR_NOT_FOUND;
}

extern "C" epic_status epic_plan_get_param(epic_plan_t p, const char* name, int* value)
{
    if (!p || !name || !value) return EPIC_ERR_INVALID_ARG;
    for (const Knob& kb : knobs_for(p)) {
        if (std::string(kb.name) != name) continue;
        *value = kb.current;
        return EPIC_OK;
    }
    p->last_error = std::string("no tuning parameter named ") + name + " on this plan's path";
    return EPIC_ERR_NOT_FOUND;
}
