// pp_batch.cu -- batched and served form: independent periodic plasmas admitted
// into slots by device-memory budget and advanced together.
//
// Each admitted context keeps its own particles, fields and stream on the
// device; pp_batch_advance enqueues up to max_steps steps of every active slot
// on that slot's stream, so the runs of different sizes overlap on the GPU,
// and records an event per slot.  Slots whose context has its own stream step
// through captured CUDA graphs (pp_set_graphs), one graph launch per step
// instead of ~25 kernel launches.  pp_batch_poll reads the event without
// blocking; a slot whose steps are all enqueued and whose event has completed
// reports PP_BATCH_DONE once and is released (its memory returns to the budget;
// the context itself stays with the caller).
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "pp_ctx.cuh"
#include "pp_internal.cuh"

using namespace pp;

struct pp_batch {
    size_t budget = 0, used = 0;
    int nslots = 0;
    struct Slot {
        pp_ctx *ctx = nullptr;
        int64_t left = 0;       // steps not yet enqueued
        int64_t done = 0;       // steps enqueued
        size_t bytes = 0;
        cudaEvent_t ev = nullptr;
        cudaEvent_t pre = nullptr;    // fused rounds: the slot's work before the shared launch
        bool busy = false;
        bool graphs_before = false;   // the context's step-graph setting before admission
        int status = PP_OK;
    } *slot = nullptr;
    // fused rounds (pp_batch_set_fused): one persistent particle launch per group
    // of compatible slots on the batch's own stream
    bool fused = false;
    cudaStream_t st = nullptr;
    cudaEvent_t join = nullptr;
    int nsm = 0;
    static constexpr int kGroups = 16;   // cells_batch_key values
    CellsBatchScratch scr[kGroups];
    void *h_args[2][kGroups] = {}, *h_items[2][kGroups] = {};   // pinned, by round parity
    size_t h_args_cap[2][kGroups] = {}, h_items_cap[2][kGroups] = {};
    cudaEvent_t h_done[2][kGroups] = {};  // the copies from h_*[parity][group] have run
    int64_t rounds = 0;
    int64_t fused_launches = 0;
    char err[256] = {0};
};

static int bfail(pp_batch *b, int code, const char *msg) {
    if (b) snprintf(b->err, sizeof b->err, "%s", msg);
    return code;
}

// Return a slot's bytes to the budget and its context to the setting it came
// with.  Only called once the context's stream holds no more of the slot's work.
static void release(pp_batch *b, pp_batch::Slot &S) {
    if (static_cast<Ctx *>(S.ctx)->use_graphs != S.graphs_before) pp_set_graphs(S.ctx, S.graphs_before ? 1 : 0);
    S.busy = false;
    S.ctx = nullptr;
    b->used -= S.bytes;
}

// Device bytes of a context on a mesh of n cells (the mirror-extended mesh
// between walls) with the given rounded species capacities: 21 padded mesh
// arrays, the compact rho and Gauss reference, and per species two particle
// buffers, the sort keys (and, in the mixed form, the permutation) and the
// per-key offsets, plus the sort's counters.
static int64_t context_bytes(const int n[3], bool fp64, int ns, const int64_t *cap) {
    int64_t padded = 1, cells = 1, nkeys = kSubKeys;
    for (int a = 0; a < 3; ++a) {
        padded *= n[a] + 2 * kGhost;
        cells *= n[a];
        const int t = n[a] < 8 ? n[a] : 8;
        nkeys *= (int64_t)((n[a] + t - 1) / t) * t;
    }
    int64_t bytes = padded * (fp64 ? 8 : 4) * 21 + 2 * 8 * cells;
    for (int s = 0; s < ns; ++s) {
        const int64_t per = fp64 ? 48 : 28;
        bytes += 2 * per * cap[s] + (fp64 ? 4 : 8) * cap[s] + 4 * (nkeys + 1);
    }
    return bytes + 4 * (nkeys + 1);
}

// Device bytes held by a context (mesh, diagnostics and particle storage).
extern "C" int64_t pp_device_bytes(pp_ctx *p) {
    if (!p) return 0;
    Ctx *c = p;
    int64_t cap[PP_MAX_SPECIES];
    for (int s = 0; s < c->nspecies; ++s) cap[s] = c->sp[s].cap;
    return context_bytes(c->g.n, c->fp64, c->nspecies, cap);
}

extern "C" int64_t pp_estimate_device_bytes(const pp_grid_desc *d, int nspecies, const int64_t *capacities) {
    if (!d || nspecies < 0 || nspecies > PP_MAX_SPECIES || (nspecies > 0 && !capacities)) return 0;
    const int bnd[3] = {d->boundary_x, d->boundary_y, d->boundary_z}, nphys[3] = {d->nx, d->ny, d->nz};
    int n[3];
    for (int a = 0; a < 3; ++a) {
        if (nphys[a] < 1) return 0;
        n[a] = bnd[a] == PP_BOUNDARY_WALLS ? 2 * nphys[a] : nphys[a];
    }
    int64_t cap[PP_MAX_SPECIES];
    for (int s = 0; s < nspecies; ++s) {
        if (capacities[s] < 0) return 0;
        cap[s] = capacities[s] == 0 ? 64 : (capacities[s] + 63) / 64 * 64;   // as pp_init_species rounds
    }
    return context_bytes(n, d->precision == PP_FP64, nspecies, cap);
}

extern "C" int pp_batch_create(pp_batch **out, int64_t budget_bytes, int max_slots) {
    if (!out || budget_bytes <= 0 || max_slots < 1 || max_slots > 4096) return PP_EINVAL;
    pp_batch *b = new (std::nothrow) pp_batch();
    if (!b) return PP_ENOMEM;
    b->budget = (size_t)budget_bytes;
    b->nslots = max_slots;
    b->slot = new (std::nothrow) pp_batch::Slot[max_slots];
    if (!b->slot) {
        delete b;
        return PP_ENOMEM;
    }
    *out = b;
    return PP_OK;
}

extern "C" int pp_batch_admit(pp_batch *b, pp_ctx *ctx, int64_t steps, int *slot_out) {
    if (!b || !ctx || steps < 0 || !slot_out) return bfail(b, PP_EINVAL, "pp_batch_admit: bad argument");
    size_t bytes = (size_t)pp_device_bytes(ctx);
    if (b->used + bytes > b->budget) return bfail(b, PP_EBUSY, "device-memory budget exhausted");
    int k = -1;
    for (int q = 0; q < b->nslots; ++q)
        if (!b->slot[q].busy) { k = q; break; }
    if (k < 0) return bfail(b, PP_EBUSY, "no free slot");
    for (int q = 0; q < b->nslots; ++q)
        if (b->slot[q].busy && b->slot[q].ctx == ctx)
            return bfail(b, PP_EINVAL, "pp_batch_admit: the context already holds a slot");
    pp_batch::Slot &S = b->slot[k];
    if (!S.ev && cudaEventCreateWithFlags(&S.ev, cudaEventDisableTiming) != cudaSuccess)
        return bfail(b, PP_ECUDA, "event creation failed");
    // slots step through captured graphs where the context has its own stream;
    // the previous setting comes back when the slot is released
    S.graphs_before = static_cast<Ctx *>(ctx)->use_graphs;
    if (static_cast<Ctx *>(ctx)->st) pp_set_graphs(ctx, 1);
    S.ctx = ctx;
    S.left = steps;
    S.done = 0;
    S.bytes = bytes;
    S.busy = true;
    S.status = PP_OK;
    b->used += bytes;
    *slot_out = k;
    return PP_OK;
}

// Device and pinned host room for a group's argument blocks and work items.
static cudaError_t ensure_room(pp_batch *b, int par, int grp, size_t abytes, size_t ibytes) {
    CellsBatchScratch &S = b->scr[grp];
    cudaError_t e = cudaSuccess;
    if (abytes > S.args_cap) {
        if (S.args) cudaFree(S.args);
        S.args = nullptr;
        S.args_cap = 0;
        if ((e = cudaMalloc(&S.args, abytes * 2)) != cudaSuccess) return e;
        S.args_cap = abytes * 2;
    }
    if (ibytes > S.items_cap) {
        if (S.items) cudaFree(S.items);
        S.items = nullptr;
        S.items_cap = 0;
        if ((e = cudaMalloc(&S.items, ibytes * 2)) != cudaSuccess) return e;
        S.items_cap = ibytes * 2;
    }
    if (!S.next && (e = cudaMalloc(&S.next, sizeof(int))) != cudaSuccess) return e;
    if (abytes > b->h_args_cap[par][grp]) {
        if (b->h_args[par][grp]) cudaFreeHost(b->h_args[par][grp]);
        b->h_args[par][grp] = nullptr;
        b->h_args_cap[par][grp] = 0;
        if ((e = cudaHostAlloc(&b->h_args[par][grp], abytes * 2, cudaHostAllocDefault)) != cudaSuccess) return e;
        b->h_args_cap[par][grp] = abytes * 2;
    }
    if (ibytes > b->h_items_cap[par][grp]) {
        if (b->h_items[par][grp]) cudaFreeHost(b->h_items[par][grp]);
        b->h_items[par][grp] = nullptr;
        b->h_items_cap[par][grp] = 0;
        if ((e = cudaHostAlloc(&b->h_items[par][grp], ibytes * 2, cudaHostAllocDefault)) != cudaSuccess) return e;
        b->h_items_cap[par][grp] = ibytes * 2;
    }
    if (!b->h_done[par][grp] && (e = cudaEventCreateWithFlags(&b->h_done[par][grp], cudaEventDisableTiming)) !=
                                     cudaSuccess)
        return e;
    return cudaSuccess;
}

// One fused round: every running slot's step, with the particle kernels of
// all of them as one persistent launch per group of compatible slots.
// Returns false (nothing enqueued) when a running slot cannot be fused.
static bool fused_round(pp_batch *b) {
    Ctx *run[4096];
    int qs[4096], n = 0;
    for (int q = 0; q < b->nslots; ++q) {
        pp_batch::Slot &S = b->slot[q];
        if (!S.busy || S.left <= 0 || S.status != PP_OK) continue;
        Ctx *c = S.ctx;
        if (!batch_fusable(c) || !c->st || cells_batch_key(*c) >= pp_batch::kGroups) return false;
        run[n] = c;
        qs[n++] = q;
    }
    if (n == 0) return false;
    // before the shared launch: each slot's sort and cleared current, on its stream
    int ok[4096];
    for (int k = 0; k < n; ++k) {
        pp_batch::Slot &S = b->slot[qs[k]];
        int rc = batch_step_pre(run[k]);
        if (rc == PP_OK && cudaEventRecord(S.pre, run[k]->st) != cudaSuccess) rc = PP_ECUDA;
        if (rc == PP_OK && cudaStreamWaitEvent(b->st, S.pre, 0) != cudaSuccess) rc = PP_ECUDA;
        ok[k] = rc == PP_OK;
        if (rc != PP_OK) S.status = rc;
    }
    // the shared launches, one per group
    const int par = (int)(b->rounds & 1);
    for (int grp = 0; grp < pp_batch::kGroups; ++grp) {
        Ctx *g[4096];
        int m = 0;
        int64_t tiles = 0;
        for (int k = 0; k < n; ++k)
            if (ok[k] && cells_batch_key(*run[k]) == grp) {
                g[m++] = run[k];
                tiles += (int64_t)run[k]->ntile[0] * run[k]->ntile[1] * run[k]->ntile[2];
            }
        if (m == 0) continue;
        cudaError_t e = ensure_room(b, par, grp, cells_args_bytes() * m, sizeof(int2) * tiles);
        // the pinned buffers of this parity were last read by the copies of two rounds ago
        if (e == cudaSuccess) e = cudaEventSynchronize(b->h_done[par][grp]);
        if (e == cudaSuccess)
            e = launch_particles_cells_batch(g, m, b->st, b->scr[grp], b->h_args[par][grp], b->h_items[par][grp],
                                             b->nsm);
        if (e == cudaSuccess) e = cudaEventRecord(b->h_done[par][grp], b->st);
        ++b->fused_launches;
        if (e != cudaSuccess) {
            snprintf(b->err, sizeof b->err, "fused particle launch: %s", cudaGetErrorString(e));
            for (int k = 0; k < n; ++k)
                if (ok[k] && cells_batch_key(*run[k]) == grp) {
                    b->slot[qs[k]].status = PP_ECUDA;
                    ok[k] = 0;
                }
        }
    }
    cudaEventRecord(b->join, b->st);
    // after it: each slot's current solve and field update, on its stream
    for (int k = 0; k < n; ++k) {
        if (!ok[k]) continue;
        pp_batch::Slot &S = b->slot[qs[k]];
        int rc = cudaStreamWaitEvent(run[k]->st, b->join, 0) == cudaSuccess ? batch_step_post(run[k]) : PP_ECUDA;
        if (rc != PP_OK) {
            S.status = rc;
            continue;
        }
        --S.left;
        ++S.done;
    }
    ++b->rounds;
    return true;
}

extern "C" int pp_batch_set_fused(pp_batch *b, int enable) {
    if (!b) return PP_EINVAL;
    if (enable && !b->st) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming) != cudaSuccess)
            return bfail(b, PP_ECUDA, "pp_batch_set_fused: stream or event creation failed");
        for (int q = 0; q < b->nslots; ++q)
            if (!b->slot[q].pre && cudaEventCreateWithFlags(&b->slot[q].pre, cudaEventDisableTiming) != cudaSuccess)
                return bfail(b, PP_ECUDA, "pp_batch_set_fused: event creation failed");
    }
    b->fused = enable != 0;
    return PP_OK;
}

extern "C" int pp_batch_advance(pp_batch *b, int max_steps) {
    if (!b || max_steps < 0) return bfail(b, PP_EINVAL, "pp_batch_advance: bad argument");
    if (b->fused) {
        int r = 0;
        for (; r < max_steps; ++r)
            if (!fused_round(b)) break;
        if (r < max_steps) {   // nothing fusable left running: the per-slot path takes the rest
            max_steps -= r;
        } else {
            for (int q = 0; q < b->nslots; ++q) {
                pp_batch::Slot &S = b->slot[q];
                if (S.busy && cudaEventRecord(S.ev, static_cast<Ctx *>(S.ctx)->st) != cudaSuccess)
                    S.status = PP_ECUDA;
            }
            return PP_OK;
        }
    }
    // one step per slot per round, so that slots interleave on the device
    for (int r = 0; r < max_steps; ++r) {
        bool any = false;
        for (int q = 0; q < b->nslots; ++q) {
            pp_batch::Slot &S = b->slot[q];
            if (!S.busy || S.left <= 0 || S.status != PP_OK) continue;
            int rc = pp_step(S.ctx, 1);
            if (rc != PP_OK) {
                S.status = rc;
                continue;
            }
            --S.left;
            ++S.done;
            any = true;
        }
        if (!any) break;
    }
    for (int q = 0; q < b->nslots; ++q) {
        pp_batch::Slot &S = b->slot[q];
        if (!S.busy) continue;
        Ctx *c = S.ctx;
        if (cudaEventRecord(S.ev, c->st) != cudaSuccess) S.status = PP_ECUDA;
    }
    return PP_OK;
}

extern "C" int pp_batch_poll(pp_batch *b, int slot, int64_t *steps_done, int *state) {
    if (!b || slot < 0 || slot >= b->nslots || !state) return bfail(b, PP_EINVAL, "pp_batch_poll: bad argument");
    pp_batch::Slot &S = b->slot[slot];
    if (!S.busy) {
        *state = PP_BATCH_FREE;
        return PP_OK;
    }
    if (steps_done) *steps_done = S.done;
    if (S.status != PP_OK) {
        // earlier steps of the slot may still run: wait for them before the
        // memory returns to the budget
        *state = PP_BATCH_FAILED;
        int st = S.status;
        cudaStreamSynchronize(static_cast<Ctx *>(S.ctx)->st);
        release(b, S);
        return st;
    }
    if (S.left > 0) {
        *state = PP_BATCH_RUNNING;
        return PP_OK;
    }
    cudaError_t e = cudaEventQuery(S.ev);
    if (e == cudaErrorNotReady) {
        *state = PP_BATCH_RUNNING;
        return PP_OK;
    }
    release(b, S);
    if (e != cudaSuccess) {
        *state = PP_BATCH_FAILED;
        return PP_ECUDA;
    }
    *state = PP_BATCH_DONE;
    return PP_OK;
}

extern "C" int pp_batch_used(pp_batch *b, int64_t *used, int *active) {
    if (!b) return PP_EINVAL;
    if (used) *used = (int64_t)b->used;
    if (active) {
        int n = 0;
        for (int q = 0; q < b->nslots; ++q) n += b->slot[q].busy ? 1 : 0;
        *active = n;
    }
    return PP_OK;
}

extern "C" const char *pp_batch_last_error(const pp_batch *b) { return b ? b->err : ""; }

extern "C" int pp_batch_destroy(pp_batch *b) {
    if (!b) return PP_OK;
    if (b->st) cudaStreamSynchronize(b->st);
    for (int q = 0; q < b->nslots; ++q) {
        if (b->slot[q].ev) cudaEventDestroy(b->slot[q].ev);
        if (b->slot[q].pre) cudaEventDestroy(b->slot[q].pre);
    }
    for (int g = 0; g < pp_batch::kGroups; ++g) {
        cudaFree(b->scr[g].args);
        cudaFree(b->scr[g].items);
        cudaFree(b->scr[g].next);
        for (int p = 0; p < 2; ++p) {
            if (b->h_args[p][g]) cudaFreeHost(b->h_args[p][g]);
            if (b->h_items[p][g]) cudaFreeHost(b->h_items[p][g]);
            if (b->h_done[p][g]) cudaEventDestroy(b->h_done[p][g]);
        }
    }
    if (b->join) cudaEventDestroy(b->join);
    if (b->st) cudaStreamDestroy(b->st);
    delete[] b->slot;
    delete b;
    return PP_OK;
}
