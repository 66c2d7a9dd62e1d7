// noalloc.cu — abm_dump_noalloc: the agent dump without any allocation.
//
// abm_dump stages its records in a device buffer that it allocates with
// cudaMalloc for every call.  Some callers cannot allow that: a per-step
// monitor or viewer hook that must not trigger cudaMalloc's implicit device
// synchronisation inside its time budget, code that runs while the caller's
// own allocator forbids new device allocations, or an embedding runtime that
// owns all device memory.  This entry point stages the records in a fixed
// file-scope device array instead and allocates nothing, on the device or on
// the host: the records are copied straight into the caller's buffer and
// sorted there in place.
//
// The array holds at most kNoAllocRecords records (3 MiB) and, like every
// __device__ variable, is held by every GPU that loads the library until the
// process exits.  All calls share it: each call clears its record counter
// first, and calls that overlap on the GPU (from several host threads or
// streams at once) race on it.
#include <algorithm>
#include <cstdio>
#include <string>

#include "../../include/abm.h"
#include "engine.cuh"

namespace abm {
bool internal_view(abm_sim* s, Buffers* B, Launch* L, cudaStream_t* stream, int32_t* sim, std::string** err,
                   int* device);
abm_status internal_cuda_fail(abm_sim* s, cudaError_t e, const char* where);
}

using namespace abm;

namespace {

constexpr uint32_t kNoAllocRecords = 131072;
constexpr int kMaxDevices = 64;

struct DumpScratch {
    unsigned int count;        // records produced by the last call
    unsigned int pad[63];
    abm_record rec[kNoAllocRecords];
};

static __device__ __align__(256) DumpScratch g_dump_scratch;

// Device address of g_dump_scratch, looked up once per device (host code
// must not use the symbol itself as a device address).
void* g_scratch_addr[kMaxDevices] = {};

__global__ void __launch_bounds__(256) k_dump_static(Buffers B, int32_t sim, DumpScratch* sc) {
    const Ctl* ctl = B.ctl;
    const uint32_t cur = ctl->cur;
    const uint32_t n = ctl->n_buf[cur];
    const SimDev& S = B.sims[sim];
    const ModelDev& Mo = B.models[S.model];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int4 pr = B.pm[cur][i];
        const uint32_t meta = (uint32_t)pr.z;
        if (meta & (M_DEAD | M_ABSORBED)) continue;
        if (sim_of(meta) != (uint32_t)sim) continue;
        const int4 p = unpack_rec(pr);
        const uint32_t sp = meta & M_SP, comp = (meta & M_COMP) >> M_COMP_SHIFT;
        const uint32_t id = (uint32_t)pr.w;
        const bool bound = meta & M_BOUND;
        const uint32_t k = atomicAdd(&sc->count, bound ? 2u : 1u);
        if (k + (bound ? 2u : 1u) > kNoAllocRecords) continue;  // counted, not written
        abm_record r;
        r.id = id;
        r.species = (uint8_t)sp;
        r.compartment = (uint8_t)comp;
        r.x = p.x;
        r.y = p.y;
        r.z = p.z;
        if (bound) {
            const uint32_t rx = (meta & M_RXN) >> M_RXN_SHIFT;
            const bool ra = meta & M_ROLE_A;
            const uint32_t par = B.apar[cur][i];
            r.flags = (uint8_t)(1u | (ra ? 4u : 0u));
            r.reaction = (uint8_t)rx;
            r.partner = par;
            sc->rec[k] = r;
            r.id = par;
            r.species = ra ? Mo.rx[rx].b : Mo.rx[rx].a;
            r.flags = (uint8_t)(2u | (ra ? 0u : 4u));
            r.partner = id;
            sc->rec[k + 1] = r;
        } else {
            r.flags = 0;
            r.reaction = 0xFF;
            r.partner = kNone;
            sc->rec[k] = r;
        }
    }
}

}  // namespace

extern "C" abm_status abm_dump_noalloc(abm_sim* s, abm_record* out, size_t cap, size_t* n_out) {
    if (!s || !n_out) return ABM_EINVAL;
    // finish queued steps and surface any sticky device error first
    const abm_status st = abm_sync(s);
    if (st != ABM_OK) return st;
    Buffers B;
    Launch L;
    cudaStream_t stream;
    int32_t sim;
    std::string* err;
    int owner = 0;
    if (!internal_view(s, &B, &L, &stream, &sim, &err, &owner)) return ABM_ESTATE;
    // the scratch array is per device: use the one of the device that holds
    // the handle's agents, which must be the current one
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev != owner || dev < 0 || dev >= kMaxDevices) {
        char buf[160];
        std::snprintf(buf, sizeof buf,
                      "abm_dump_noalloc: the handle lives on device %d but device %d is current", owner, dev);
        *err = buf;
        return ABM_EDEVICE;
    }
    if (!g_scratch_addr[dev]) {  // set-up, once per device, with that device current
        void* addr = nullptr;
        e = cudaGetSymbolAddress(&addr, g_dump_scratch);
        if (e != cudaSuccess || !addr)
            return internal_cuda_fail(s, e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                                      "abm_dump_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[dev] = addr;
    }
    DumpScratch* sc = static_cast<DumpScratch*>(g_scratch_addr[dev]);
    unsigned int count = 0;
    e = cudaMemsetAsync(&sc->count, 0, sizeof(unsigned int), stream);
    if (e == cudaSuccess) {
        k_dump_static<<<L.blocks_agents, 256, 0, stream>>>(B, sim, sc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&count, &sc->count, sizeof count, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return internal_cuda_fail(s, e, "abm_dump_noalloc");
    *n_out = count;
    if (count > kNoAllocRecords) {
        char buf[192];
        std::snprintf(buf, sizeof buf,
                      "abm_dump_noalloc: %u records exceed its fixed scratch of %u records; use abm_dump",
                      count, kNoAllocRecords);
        *err = buf;
        return ABM_ECAPACITY;
    }
    if (!out) return ABM_OK;  // size query
    if (cap < count) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "abm_dump_noalloc: output holds %zu records, %u needed", cap, count);
        *err = buf;
        return ABM_EINVAL;
    }
    e = cudaMemcpyAsync(out, sc->rec, (size_t)count * sizeof(abm_record), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return internal_cuda_fail(s, e, "abm_dump_noalloc: copy");
    std::sort(out, out + count, [](const abm_record& a, const abm_record& b) { return a.id < b.id; });
    return ABM_OK;
}
