// Serving loop: continuous batching of whole-image render requests over
// several device-resident grids (inference rendering of colour and depth,
// Sec. 4.2 of arXiv 2305.13220).
//
// A host scheduler thread
//   * admits queued requests (FIFO) while request slots and the device-memory
//     budget allow (outputs are carved from one pre-allocated pool),
//   * cuts admitted requests into chunks of chunk_rays pixels and packs
//     chunks of different requests, resolutions and scenes (with samples per
//     ray in the same class) into batches of at most max_batch_rays rays,
//   * launches each batch on the next of n_streams streams (at most two
//     batches in flight per stream), so batches overlap on the device while
//     new requests join the following batch as soon as they are admitted,
//   * completes a request when the events of all batches holding its chunks
//     have fired.
// Each ray is generated in the kernels from its request's camera and pixel
// index: a traversal pass (one thread per ray) writes the allocated cells it
// crosses, then the records kernel renders it with the same per-ray program
// as sdg_render_forward (a ray crossing more than kWalkCap cells is walked
// in-warp by a third kernel over the overflow list), so a request's result
// does not depend on its batch mates.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"
#include "render_core.cuh"

using namespace sdg;

namespace {

struct ChunkDesc {
    float K[4];
    float T[12];
    float tnear, tfar;
    float *rgb, *depth, *opac;
    int64_t pix0;
    int32_t npix, W, scene, N;
    uint32_t seed;
    int32_t strat;
};

// The ray of batch slot `slot` (chunk slot / chunk_rays, its pixel slot % chunk_rays); false past the chunk's end.
__device__ __forceinline__ bool slot_ray(const ChunkDesc* chunks, int chunk_rays, int64_t slot, const ChunkDesc*& ch,
                                         int64_t& pix, float3& o, float3& d) {
    const int local = (int)(slot % chunk_rays);
    ch = chunks + slot / chunk_rays;
    if (local >= ch->npix) return false;
    pix = ch->pix0 + local;
    pinhole_ray(ch->K, ch->T, (int)(pix % ch->W), (int)(pix / ch->W), o, d);
    return true;
}

// Traversal pass of a batch: one thread per ray slot.
__global__ void __launch_bounds__(256) k_serve_walk(const GridDev* __restrict__ scenes,
                                                     const ChunkDesc* __restrict__ chunks, int chunk_rays,
                                                     int64_t nslots, WalkBufs w) {
    const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= nslots) return;
    const ChunkDesc* ch;
    int64_t pix;
    float3 o, d;
    if (!slot_ray(chunks, chunk_rays, slot, ch, pix, o, d)) return;  // never rendered: no header needed
    walk_ray_records(scenes[ch->scene], o, d, ch->tnear, ch->tfar, w, slot);
}

// The ray of batch slot `slot` rendered by one warp: from the traversal pass's records, RPL per lane (OVER false),
// or walked in-warp (OVER true).
template <bool BF16, int Q, bool OVER, int RPL = 1>
__device__ __forceinline__ void serve_ray(const GridDev* scenes, const ChunkDesc* chunks, int chunk_rays,
                                          const WalkBufs& wb, int64_t slot, WarpSmem& sm, int lane) {
    const ChunkDesc* ch;
    RayJob j;
    if (!slot_ray(chunks, chunk_rays, slot, ch, j.idx, j.o, j.d)) return;  // warp-uniform
    j.tn = ch->tnear;
    j.tf = ch->tfar;
    j.ray_id = (uint32_t)j.idx;
    j.slot = slot;
    PassArgs a{};
    a.N = ch->N;
    a.seed = ch->seed;
    a.strat = ch->strat;
    a.n = 0;
    a.out_rgb = ch->rgb;
    a.out_depth = ch->depth;
    a.out_opac = ch->opac;
    a.walk = wb;
    ray_program<PASS_FWD, BF16, 0, Q, OVER, RPL>(scenes[ch->scene], a, j, sm, lane);
}

// One warp per slot of the batch, cells from the traversal pass's records (a slot without records is left to
// k_serve_rest).  Blocks of kServeWarps warps, 6 per SM at 4 samples per lane (80 registers), 4 above.
constexpr int kServeWarps = 4;

template <bool BF16, int Q>
__global__ void __launch_bounds__(32 * kServeWarps, (Q <= 4 ? 6 : 4))
    k_serve(const GridDev* __restrict__ scenes, const ChunkDesc* __restrict__ chunks, int chunk_rays, WalkBufs wb) {
    __shared__ WarpSmem smem[1];
    const int64_t slot = (int64_t)blockIdx.x * kServeWarps + (threadIdx.x >> 5);
    serve_ray<BF16, Q, false>(scenes, chunks, chunk_rays, wb, slot, smem[0], threadIdx.x & 31);
}

// The batch's rays beyond the records kernel: the mid list (kWalkCap + 1 .. kWalkSlot allocated cells, from their
// records two per lane), then the overflow list (more cells, walked in-warp), by a grid of at most
// kServeRestBlocks blocks striding over them; it runs alone after the records kernel on the batch's stream, so it
// takes the registers that keep the loops free of spills (2 blocks per SM).
constexpr unsigned kServeRestBlocks = 296;

template <bool BF16, int Q>
__global__ void __launch_bounds__(256, 2)
    k_serve_rest(const GridDev* __restrict__ scenes, const ChunkDesc* __restrict__ chunks, int chunk_rays,
                 WalkBufs wb) {
    __shared__ WarpSmem smem[kWarpsPerBlock];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n_mid = (int64_t)__ldg(wb.n_mid), n_over = (int64_t)__ldg(wb.n_over);
    const int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + warp, stride = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t q = w; q < n_mid; q += stride)
        serve_ray<BF16, Q, false, 2>(scenes, chunks, chunk_rays, wb, __ldg(wb.mid + q), smem[warp], lane);
    for (int64_t q = w; q < n_over; q += stride)
        serve_ray<BF16, Q, true>(scenes, chunks, chunk_rays, wb, __ldg(wb.over + q), smem[warp], lane);
}

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over one device pool, 256-byte granules, coalescing frees.
struct Pool {
    char* base = nullptr;
    int64_t size = 0;
    std::map<int64_t, int64_t> free_;  // offset -> length
    int64_t in_use = 0, peak = 0;
    void init(char* b, int64_t n) {
        base = b;
        size = n;
        free_.clear();
        free_[0] = n;
    }
    int64_t alloc(int64_t n) {
        n = (n + 255) & ~(int64_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= n) {
                int64_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > n) free_[off + n] = len - n;
                in_use += n;
                if (in_use > peak) peak = in_use;
                return off;
            }
        return -1;
    }
    void release(int64_t off, int64_t n) {
        n = (n + 255) & ~(int64_t)255;
        in_use -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

enum ReqState { QUEUED = 0, ADMITTED = 1, DONE = 2 };

struct Req {
    sdg_request q;
    int state = QUEUED;
    bool cancel = false;
    int64_t off = -1, bytes = 0;
    float *rgb = nullptr, *depth = nullptr, *opac = nullptr;
    int64_t npix = 0, next_pix = 0;
    int pending = 0;  // launched batches not yet complete that hold chunks of this request
    double t_submit = 0, t_admit = 0, t_done = 0;
};

struct Batch {
    cudaStream_t stream;
    int stream_index = 0;
    cudaEvent_t ev;
    ChunkDesc* h_chunks = nullptr;
    ChunkDesc* d_chunks = nullptr;
    GridDev* h_scenes = nullptr;
    GridDev* d_scenes = nullptr;
    std::vector<uint64_t> tickets;
    bool busy = false;
    int64_t rays = 0;
};

int pick_q(int N) { return N <= 64 ? 2 : N <= 128 ? 4 : N <= 192 ? 6 : 8; }

}  // namespace

struct sdg_server_s {
    sdg_server_opts o;
    std::vector<sdg_grid> scenes;
    bool bf16 = false;
    char* pool_mem = nullptr;
    Pool pool;
    std::vector<cudaStream_t> streams;
    std::vector<WalkBufs> walk;  // traversal records of the batch running on each stream (max_batch_rays slots)
    std::vector<Batch> batches;
    std::deque<Batch*> inflight;  // launch order
    int next_stream = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::deque<uint64_t> queue;
    std::vector<uint64_t> active;  // admitted, not yet fully launched or completed
    std::unordered_map<uint64_t, Req> reqs;
    int in_flight = 0;
    sdg_server_stats st{};
    std::string worker_error;

    void free_request_memory(Req& r) {
        if (r.off >= 0) pool.release(r.off, r.bytes);
        r.off = -1;
    }

    // All four scheduler steps run with mu held.
    bool reap() {
        bool any = false;
        while (!inflight.empty()) {
            Batch* b = inflight.front();
            cudaError_t e = cudaEventQuery(b->ev);
            if (e == cudaErrorNotReady) break;
            if (e != cudaSuccess) worker_error = cudaGetErrorString(e);
            inflight.pop_front();
            const double t = now_ms();
            for (uint64_t tk : b->tickets) {
                auto it = reqs.find(tk);
                if (it == reqs.end()) continue;
                Req& r = it->second;
                if (--r.pending == 0 && r.next_pix >= r.npix) {
                    r.state = DONE;
                    r.t_done = t;
                    --in_flight;
                    ++st.completed;
                    if (r.cancel) {
                        free_request_memory(r);
                        reqs.erase(it);
                    }
                }
            }
            b->tickets.clear();
            b->busy = false;
            any = true;
        }
        if (any) cv.notify_all();
        return any;
    }

    bool admit() {
        bool any = false;
        while (!queue.empty() && in_flight < o.max_slots) {
            Req& r = reqs[queue.front()];
            int64_t off = pool.alloc(r.bytes);
            if (off < 0) break;  // head of line waits for memory
            r.off = off;
            float* base = reinterpret_cast<float*>(pool_mem + off);
            r.rgb = base;
            r.depth = base + 3 * r.npix;
            r.opac = base + 4 * r.npix;
            r.state = ADMITTED;
            r.t_admit = now_ms();
            active.push_back(queue.front());
            queue.pop_front();
            ++in_flight;
            ++st.admitted;
            any = true;
        }
        return any;
    }

    Batch* free_batch() {
        for (auto& b : batches)
            if (!b.busy) return &b;
        return nullptr;
    }

    int launch() {
        int launched = 0;
        const int max_chunks = o.max_batch_rays / o.chunk_rays;
        while (!active.empty()) {
            Batch* b = free_batch();
            if (!b) break;
            int nch = 0, maxN = 1;
            // One batch = one sample-slot class (Q = ceil(N/32) rounded as the kernels are built), so that
            // every request runs the same kernel instantiation alone or in any mix: its rays' arithmetic,
            // and hence its result, do not depend on its batch mates.
            const int qclass = pick_q(reqs[active.front()].q.n_samples);
            // oldest admitted requests first; a request contributes chunks until the batch is full
            for (size_t i = 0; i < active.size() && nch < max_chunks; ++i) {
                Req& r = reqs[active[i]];
                if (pick_q(r.q.n_samples) != qclass) continue;
                bool used = false;
                while (r.next_pix < r.npix && nch < max_chunks) {
                    ChunkDesc& c = b->h_chunks[nch++];
                    std::memcpy(c.K, r.q.K, sizeof(c.K));
                    std::memcpy(c.T, r.q.Twc, sizeof(c.T));
                    c.tnear = r.q.tnear;
                    c.tfar = r.q.tfar;
                    c.rgb = r.rgb;
                    c.depth = r.depth;
                    c.opac = r.opac;
                    c.pix0 = r.next_pix;
                    c.npix = (int32_t)std::min<int64_t>(o.chunk_rays, r.npix - r.next_pix);
                    c.W = r.q.W;
                    c.scene = r.q.scene_id;
                    c.N = r.q.n_samples;
                    c.seed = r.q.seed;
                    c.strat = r.q.stratified;
                    r.next_pix += c.npix;
                    b->rays += c.npix;
                    maxN = std::max(maxN, (int)r.q.n_samples);
                    used = true;
                }
                if (used) {
                    ++r.pending;
                    b->tickets.push_back(active[i]);
                }
            }
            if (nch == 0) break;
            // drop fully launched requests from the active list
            std::vector<uint64_t> keep;
            for (uint64_t tk : active)
                if (reqs[tk].next_pix < reqs[tk].npix) keep.push_back(tk);
            active.swap(keep);
            for (size_t s = 0; s < scenes.size(); ++s) b->h_scenes[s] = scenes[s]->dev();
            b->stream_index = next_stream;
            b->stream = streams[next_stream];
            next_stream = (next_stream + 1) % (int)streams.size();
            cudaMemcpyAsync(b->d_scenes, b->h_scenes, sizeof(GridDev) * scenes.size(), cudaMemcpyHostToDevice,
                            b->stream);
            cudaMemcpyAsync(b->d_chunks, b->h_chunks, sizeof(ChunkDesc) * nch, cudaMemcpyHostToDevice, b->stream);
            // batches on one stream run in order, so the stream's records serve each in turn
            const WalkBufs& wb = walk[b->stream_index];
            const int64_t nslots = (int64_t)nch * o.chunk_rays;
            const unsigned blocks = (unsigned)((nslots + kWarpsPerBlock - 1) / kWarpsPerBlock);
            const int Q = pick_q(maxN);
            cudaMemsetAsync(wb.n_over, 0, 2 * sizeof(int), b->stream);  // n_over and n_mid
            k_serve_walk<<<(unsigned)((nslots + 255) / 256), 256, 0, b->stream>>>(b->d_scenes, b->d_chunks,
                                                                                   o.chunk_rays, nslots, wb);
#define SDG_SERVE(BF, QQ)                                                                                      \
    do {                                                                                                       \
        k_serve<BF, QQ><<<(unsigned)((nslots + kServeWarps - 1) / kServeWarps), 32 * kServeWarps, 0, b->stream>>>(  \
            b->d_scenes, b->d_chunks, o.chunk_rays, wb);                                                       \
        k_serve_rest<BF, QQ><<<std::min(blocks, kServeRestBlocks), 256, 0, b->stream>>>(                        \
            b->d_scenes, b->d_chunks, o.chunk_rays, wb);                                                       \
    } while (0)
            if (bf16) {
                if (Q == 2) SDG_SERVE(true, 2); else if (Q == 4) SDG_SERVE(true, 4);
                else if (Q == 6) SDG_SERVE(true, 6); else SDG_SERVE(true, 8);
            } else {
                if (Q == 2) SDG_SERVE(false, 2); else if (Q == 4) SDG_SERVE(false, 4);
                else if (Q == 6) SDG_SERVE(false, 6); else SDG_SERVE(false, 8);
            }
#undef SDG_SERVE
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) worker_error = cudaGetErrorString(e);
            cudaEventRecord(b->ev, b->stream);
            b->busy = true;
            inflight.push_back(b);
            ++st.launches;
            st.rays_rendered += b->rays;
            b->rays = 0;
            ++launched;
        }
        return launched;
    }

    void loop() {
        cudaSetDevice(o.device);
        std::unique_lock<std::mutex> lk(mu);
        while (!stop) {
            bool progress = reap();
            progress |= admit();
            progress |= launch() > 0;
            if (!progress) {
                if (inflight.empty() && queue.empty() && active.empty())
                    cv.wait_for(lk, std::chrono::milliseconds(5));
                else
                    cv.wait_for(lk, std::chrono::microseconds(20));
            }
        }
    }
};

static void free_walk(sdg_server s) {
    for (WalkBufs& w : s->walk) {
        void* ptrs[] = {w.hdr, w.s0, w.rec, w.over};
        for (void* p : ptrs)
            if (p) cudaFree(p);
    }
    s->walk.clear();
}

extern "C" int sdg_server_create(const sdg_server_opts* o, sdg_server* out) {
    if (!o || !out) return fail(SDG_ERR_ARG, "sdg_server_create: null argument");
    *out = nullptr;
    if (o->hbm_budget_bytes < 4096 || o->max_slots < 1 || o->n_streams < 1 || o->n_streams > 8 ||
        o->chunk_rays < 32 || o->chunk_rays % 32 || o->max_batch_rays < o->chunk_rays ||
        o->max_batch_rays % o->chunk_rays || o->reserved != 0)
        return fail(SDG_ERR_ARG, "sdg_server_create: invalid options");
    SDG_CUDA_TRY(cudaSetDevice(o->device));
    sdg_server s = new (std::nothrow) sdg_server_s();
    if (!s) return fail(SDG_ERR_OOM, "host allocation");
    s->o = *o;
    auto cleanup = [&](int rc) {
        std::string m = sdg_last_error();
        for (auto& b : s->batches) {
            if (b.ev) cudaEventDestroy(b.ev);
            if (b.h_chunks) cudaFreeHost(b.h_chunks);
            if (b.d_chunks) cudaFree(b.d_chunks);
            if (b.h_scenes) cudaFreeHost(b.h_scenes);
            if (b.d_scenes) cudaFree(b.d_scenes);
        }
        for (auto st : s->streams) cudaStreamDestroy(st);
        free_walk(s);
        if (s->pool_mem) cudaFree(s->pool_mem);
        delete s;
        return fail(rc, m);
    };
    cudaError_t e = cudaMalloc((void**)&s->pool_mem, o->hbm_budget_bytes);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "server pool"));
    s->pool.init(s->pool_mem, o->hbm_budget_bytes);
    for (int i = 0; i < o->n_streams; ++i) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "server stream"));
        s->streams.push_back(st);
        // traversal records for max_batch_rays slots: 8 + kWalkSlot * 20 bytes a slot, the overflow and mid lists
        // and their lengths (one allocation: over [R], mid [R], n_over, n_mid)
        const int64_t R = o->max_batch_rays;
        WalkBufs w{};
        if ((e = cudaMalloc((void**)&w.hdr, sizeof(int2) * R)) != cudaSuccess ||
            (e = cudaMalloc((void**)&w.s0, sizeof(float) * kWalkSlot * R)) != cudaSuccess ||
            (e = cudaMalloc((void**)&w.rec, sizeof(int4) * kWalkSlot * R)) != cudaSuccess ||
            (e = cudaMalloc((void**)&w.over, sizeof(int) * (2 * R + 2))) != cudaSuccess) {
            s->walk.push_back(w);
            return cleanup(cuda_fail(e, "server traversal records"));
        }
        w.mid = w.over + R;
        w.n_over = w.over + 2 * R;
        w.n_mid = w.over + 2 * R + 1;
        s->walk.push_back(w);
    }
    const int max_chunks = o->max_batch_rays / o->chunk_rays;
    s->batches.resize(2 * o->n_streams);
    for (auto& b : s->batches) {
        b.ev = nullptr;
        if ((e = cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaMallocHost((void**)&b.h_chunks, sizeof(ChunkDesc) * max_chunks)) != cudaSuccess ||
            (e = cudaMalloc((void**)&b.d_chunks, sizeof(ChunkDesc) * max_chunks)) != cudaSuccess)
            return cleanup(cuda_fail(e, "server batch buffers"));
    }
    s->worker = std::thread([s] { s->loop(); });
    *out = s;
    return SDG_OK;
}

extern "C" int sdg_server_add_scene(sdg_server s, sdg_grid g, int32_t* id) {
    if (!s || !g || !id) return fail(SDG_ERR_ARG, "sdg_server_add_scene: null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->next_ticket != 1) return fail(SDG_ERR_ARG, "sdg_server_add_scene: scenes must be added before requests");
    if (g->device != s->o.device) return fail(SDG_ERR_ARG, "sdg_server_add_scene: grid on another device");
    const bool bf = g->desc.rgb_dtype == SDG_BF16;
    if (!s->scenes.empty() && bf != s->bf16) return fail(SDG_ERR_ARG, "sdg_server_add_scene: mixed colour layouts");
    if (!s->scenes.empty() && g->desc.n_sem != s->scenes[0]->desc.n_sem)
        return fail(SDG_ERR_ARG, "sdg_server_add_scene: mixed semantic channel counts");
    {
        // from now on the grid's block structure is fixed (activation and destruction return SDG_ERR_BUSY), so
        // the scheduler may snapshot its descriptor without its lock
        std::lock_guard<std::mutex> gl(g->mu);
        ++g->served;
    }
    s->bf16 = bf;
    s->scenes.push_back(g);
    const size_t n = s->scenes.size();
    for (auto& b : s->batches) {
        if (b.h_scenes) cudaFreeHost(b.h_scenes);
        if (b.d_scenes) cudaFree(b.d_scenes);
        b.h_scenes = nullptr;
        b.d_scenes = nullptr;
        SDG_CUDA_TRY(cudaMallocHost((void**)&b.h_scenes, sizeof(GridDev) * n));
        SDG_CUDA_TRY(cudaMalloc((void**)&b.d_scenes, sizeof(GridDev) * n));
    }
    *id = (int32_t)(n - 1);
    return SDG_OK;
}

extern "C" int sdg_server_submit(sdg_server s, const sdg_request* q, uint64_t* ticket) {
    if (!s || !q || !ticket) return fail(SDG_ERR_ARG, "sdg_server_submit: null argument");
    if (q->H <= 0 || q->W <= 0 || q->n_samples < 1 || q->n_samples > 256 || !(q->K[0] != 0.f) || !(q->K[1] != 0.f))
        return fail(SDG_ERR_ARG, "sdg_server_submit: invalid request");
    const int64_t npix = (int64_t)q->H * q->W;
    const int64_t bytes = ((npix * 5 * (int64_t)sizeof(float)) + 255) & ~(int64_t)255;
    if (bytes > s->o.hbm_budget_bytes)
        return fail(SDG_ERR_CAPACITY, "sdg_server_submit: request outputs exceed the server's memory budget");
    std::lock_guard<std::mutex> lk(s->mu);
    if (q->scene_id < 0 || q->scene_id >= (int)s->scenes.size())
        return fail(SDG_ERR_ARG, "sdg_server_submit: invalid scene_id");
    if (!s->worker_error.empty()) return fail(SDG_ERR_CUDA, "server: " + s->worker_error);
    uint64_t tk = s->next_ticket++;
    Req& r = s->reqs[tk];
    r.q = *q;
    r.npix = npix;
    r.bytes = bytes;
    r.t_submit = now_ms();
    s->queue.push_back(tk);
    ++s->st.submitted;
    *ticket = tk;
    s->cv.notify_all();
    return SDG_OK;
}

static void fill_result(const Req& r, sdg_result* out) {
    out->status = SDG_OK;
    out->H = r.q.H;
    out->W = r.q.W;
    out->rgb = r.rgb;
    out->depth = r.depth;
    out->opac = r.opac;
    out->t_submit_ms = r.t_submit;
    out->t_admit_ms = r.t_admit;
    out->t_done_ms = r.t_done;
}

extern "C" int sdg_server_poll(sdg_server s, uint64_t ticket, sdg_result* out) {
    if (!s || !out) return fail(SDG_ERR_ARG, "sdg_server_poll: null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end() || it->second.cancel) return fail(SDG_ERR_NOT_FOUND, "unknown ticket");
    if (it->second.state != DONE) {
        out->status = SDG_ERR_BUSY;
        return SDG_ERR_BUSY;
    }
    fill_result(it->second, out);
    return SDG_OK;
}

extern "C" int sdg_server_wait(sdg_server s, uint64_t ticket, int64_t timeout_ms, sdg_result* out) {
    if (!s || !out) return fail(SDG_ERR_ARG, "sdg_server_wait: null argument");
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (true) {
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end() || it->second.cancel) return fail(SDG_ERR_NOT_FOUND, "unknown ticket");
        if (it->second.state == DONE) {
            fill_result(it->second, out);
            return SDG_OK;
        }
        if (!s->worker_error.empty()) return fail(SDG_ERR_CUDA, "server: " + s->worker_error);
        if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout) {
            auto it2 = s->reqs.find(ticket);
            if (it2 != s->reqs.end() && it2->second.state == DONE) {
                fill_result(it2->second, out);
                return SDG_OK;
            }
            out->status = SDG_ERR_TIMEOUT;
            return fail(SDG_ERR_TIMEOUT, "sdg_server_wait: request not done before the deadline");
        }
    }
}

extern "C" int sdg_server_release(sdg_server s, uint64_t ticket) {
    if (!s) return fail(SDG_ERR_ARG, "sdg_server_release: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end() || it->second.cancel) return fail(SDG_ERR_NOT_FOUND, "unknown ticket");
    Req& r = it->second;
    if (r.state == QUEUED) {
        for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
            if (*q == ticket) {
                s->queue.erase(q);
                break;
            }
        s->reqs.erase(it);
    } else if (r.state == DONE) {
        s->free_request_memory(r);
        s->reqs.erase(it);
    } else {
        r.cancel = true;  // freed by the scheduler when its last batch completes
    }
    s->cv.notify_all();
    return SDG_OK;
}

extern "C" int sdg_server_get_stats(sdg_server s, sdg_server_stats* st) {
    if (!s || !st) return fail(SDG_ERR_ARG, "sdg_server_get_stats: null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *st = s->st;
    st->bytes_in_use = s->pool.in_use;
    st->peak_bytes_in_use = s->pool.peak;
    st->in_flight = s->in_flight;
    st->queued = (int32_t)s->queue.size();
    return SDG_OK;
}

extern "C" int sdg_server_destroy(sdg_server s) {
    if (!s) return SDG_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->o.device);
    for (auto st : s->streams) cudaStreamSynchronize(st);
    for (auto& b : s->batches) {
        if (b.ev) cudaEventDestroy(b.ev);
        if (b.h_chunks) cudaFreeHost(b.h_chunks);
        if (b.d_chunks) cudaFree(b.d_chunks);
        if (b.h_scenes) cudaFreeHost(b.h_scenes);
        if (b.d_scenes) cudaFree(b.d_scenes);
    }
    for (auto st : s->streams) cudaStreamDestroy(st);
    free_walk(s);
    if (s->pool_mem) cudaFree(s->pool_mem);
    for (sdg_grid g : s->scenes) {
        std::lock_guard<std::mutex> gl(g->mu);
        --g->served;
    }
    delete s;
    return SDG_OK;
}
