// batch.cu -- many independent FP32 runs of uneven grid size advanced
// together: one kernel launch per RK stage over a shared tile queue, per-run
// CFL steps, CUDA-graph replay of whole batch steps, and an autotuner over
// the launch configuration.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "sac_ctx.h"
#include "stage_fp32.cuh"

using namespace sac;

namespace {

struct RunCtl {
    DevScalars* sc;
    double dx, dy, courant;
};

struct BatchArgs {
    const StageArgs<float>* args;   // [nruns][4]: arguments of each run for stage 1..4
    const int4* tiles;              // queue order: (run, tile x, tile y, 0)
    int ntiles;
    unsigned* counters;             // [4] per-stage queue heads (persistent mode)
    int persistent;
    const CUtensorMap* tmaps;       // [nruns][4]: tensor map of each run's stage input, or null
};

// Start one step of every run; also re-arms the four stage queues.
__global__ void batch_begin_kernel(const RunCtl* __restrict__ ctl, int n, unsigned* counters)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 4) counters[i] = 0u;
    if (i < n) step_begin(ctl[i].sc, ctl[i].dx, ctl[i].dy, ctl[i].courant, 1, 0.0);
}

// Copy the arguments of run `run`, stage STAGE, into shared memory (all threads).
template <int STAGE>
__device__ __forceinline__ void load_args(const BatchArgs& b, int run, StageArgs<float>& dst)
{
    const int* src = reinterpret_cast<const int*>(&b.args[run * 4 + (STAGE - 1)]);
    int* d = reinterpret_cast<int*>(&dst);
    for (int k = threadIdx.x; k < (int)(sizeof(StageArgs<float>) / sizeof(int)); k += blockDim.x) d[k] = src[k];
}

template <class G, int STAGE, bool BG, bool HD>
__global__ void __launch_bounds__(G::NT, G::MINB) stage_fp32_batch(const BatchArgs b)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ unsigned long long red[2][G::NW];
    // current / next tile's run (raw storage: StageArgs has member initialisers,
    // and the arguments are always copied in by load_args)
    __shared__ __align__(16) unsigned char sa_raw[2 * sizeof(StageArgs<float>)];
    StageArgs<float>* sa = reinterpret_cast<StageArgs<float>*>(sa_raw);
    __shared__ int tile_s[2];
    __shared__ int run_s[2], skip_s[2], coef_s;   // run whose arguments sa[k] hold, its skip flag; run of S.ax/S.ay
    __shared__ __align__(8) unsigned long long bar;   // staging completion (persistent mode)
    f32k::Smem<G>& S = *reinterpret_cast<f32k::Smem<G>*>(smem_raw);
    if (!b.persistent) {
        // one tile per CTA: stage inside the tile
        const int t = blockIdx.x;
        if (t >= b.ntiles) return;
        const int4 d = b.tiles[t];
        load_args<STAGE>(b, d.x, sa[0]);
        __syncthreads();
        if (!sa[0].sc->skip) {
            f32k::store_hd_coeffs(sa[0], S, threadIdx.x);   // visible after the tile's staging barrier
            const f32k::StepConsts K = f32k::load_step_consts(sa[0].sc);
            unsigned long long m[2] = {0ull, 0ull};
            f32k::tile_body<G, STAGE, BG, HD, false, false>(sa[0], d.y * G::TX, d.z * G::TY, S, K, m);
            if (STAGE == 4) f32k::block_speed_max(m, red, sa[0].sc);
        }
        return;
    }
    // persistent: tiles from the queue; the next tile is fetched when a tile
    // starts so that its region streams into shared memory (one TMA tensor copy
    // per plane with the next run's tensor map, else bulk row copies) during the
    // current tile's Y sweep.  persistent == 1 takes tiles from an atomic queue
    // head; persistent == 2 walks the queue with a fixed stride (tile
    // blockIdx.x + k * gridDim.x), so the next index needs no atomic round trip.
    // A run's arguments are reloaded only when the run changes, and stage 4
    // folds its signal-speed maximum into the run's key once per run change.
    const bool tma = b.tmaps != nullptr && (f32k::smem_u32(&S.u[0][0][0]) & 127u) == 0;
    const bool strided = b.persistent == 2;
    const auto tmap = [&](int run) { return tma ? &b.tmaps[run * 4 + (STAGE - 1)] : nullptr; };
    if (threadIdx.x == 0) {
        f32k::mbar_init(&bar, 1);
        if (!strided) tile_s[0] = (int)atomicAdd(&b.counters[STAGE - 1], 1u);
    }
    __syncthreads();
    int nxt = strided ? (int)blockIdx.x : tile_s[0], buf = 0;
    unsigned phase = 0;
    bool failed = false;
    if (nxt >= b.ntiles) return;
    int4 d = b.tiles[nxt];
    load_args<STAGE>(b, d.x, sa[0]);
    __syncthreads();
    bool staged = !sa[0].sc->skip;
    if (threadIdx.x == 0) { run_s[0] = d.x; skip_s[0] = !staged; run_s[1] = -1; coef_s = -1; }
    unsigned long long m[2] = {0ull, 0ull};
    if (staged) {
        f32k::NextTile first = f32k::next_tile(sa[0], true, d.y * G::TX, d.z * G::TY);
        first.tm = tmap(d.x);
        if (threadIdx.x == 0)
            f32k::mbar_expect_tx(&bar, first.tm ? f32k::tile_bytes_tm<G>() : f32k::tile_bytes<G>());
#pragma unroll
        for (int p = 0; p < 3; ++p) f32k::stage_plane_bulk(first, S, p, &bar);
    }
    __syncthreads();   // run_s, skip_s, coef_s set (later updates are ordered by the loop's barriers)
    while (true) {
        if (strided) {
            nxt += (int)gridDim.x;
        } else {
            if (threadIdx.x == 0) tile_s[buf ^ 1] = (int)atomicAdd(&b.counters[STAGE - 1], 1u);
            __syncthreads();
            nxt = tile_s[buf ^ 1];
        }
        int4 dn = make_int4(-1, 0, 0, 0);
        bool reload = false;
        if (nxt < b.ntiles) {
            dn = b.tiles[nxt];
            reload = run_s[buf ^ 1] != dn.x;
            if (reload) load_args<STAGE>(b, dn.x, sa[buf ^ 1]);
        }
        const bool coef = coef_s != d.x;
        __syncthreads();
        const int skip_n = reload ? sa[buf ^ 1].sc->skip : skip_s[buf ^ 1];
        if (threadIdx.x == 0) {
            if (reload) { run_s[buf ^ 1] = dn.x; skip_s[buf ^ 1] = skip_n; }
            if (staged) coef_s = d.x;
        }
        const StageArgs<float>& A = sa[buf];
        const bool nstage = nxt < b.ntiles && !skip_n;
        f32k::NextTile nt = f32k::next_tile(sa[buf ^ 1], nstage, dn.y * G::TX, dn.z * G::TY);
        nt.tm = nstage ? tmap(dn.x) : nullptr;
        if (staged) {
            if (coef) f32k::store_hd_coeffs(A, S, threadIdx.x);   // visible after the tile's staging barrier
            const f32k::StepConsts K = f32k::load_step_consts(A.sc);
            f32k::tile_body<G, STAGE, BG, HD, true, false>(A, d.y * G::TX, d.z * G::TY, S, K, m, nt,
                                                          &bar, &phase, &failed);
            if (failed) return;
            // the next tile belongs to another run (or there is none): fold this run's
            // maximum now; a later tile of the same run folds again (atomicMax)
            if (STAGE == 4 && dn.x != d.x) {
                f32k::block_speed_max(m, red, A.sc);
                m[0] = m[1] = 0ull;
            }
        } else if (nstage) {
            // this tile's run is done or failed: nothing was staged for it, so
            // the next tile's region is copied now
            if (threadIdx.x == 0) f32k::mbar_expect_tx(&bar, nt.tm ? f32k::tile_bytes_tm<G>() : f32k::tile_bytes<G>());
#pragma unroll
            for (int p = 0; p < 3; ++p) f32k::stage_plane_bulk(nt, S, p, &bar);
        }
        if (nxt >= b.ntiles) break;
        staged = nstage;
        d = dn;
        buf ^= 1;
        __syncthreads();   // sa[buf ^ 1] is rewritten by the next iteration
    }
}

// Ghost frames of every run's stage output (one grid row per run).
__global__ void halo_fp32_batch(const StageArgs<float>* __restrict__ args, int stage)
{
    const StageArgs<float>& a = args[blockIdx.y * 4 + (stage - 1)];
    if (a.sc->skip || (a.bc_x == BC_FIXED && a.bc_y == BC_FIXED)) return;
    const long long n = f32k::halo_count(a.L);
    float2* w = reinterpret_cast<float2*>(a.sout);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        f32k::halo_cell(w, a.L, a.bc_x, a.bc_y, t);
}

template <class G, int S, bool BG, bool HD>
cudaError_t set_attr()
{
    return cudaFuncSetAttribute(stage_fp32_batch<G, S, BG, HD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(f32k::Smem<G>));
}

template <class G, bool BG, bool HD>
cudaError_t attr_all()
{
    cudaError_t e = set_attr<G, 1, BG, HD>();
    if (e == cudaSuccess) e = set_attr<G, 2, BG, HD>();
    if (e == cudaSuccess) e = set_attr<G, 3, BG, HD>();
    if (e == cudaSuccess) e = set_attr<G, 4, BG, HD>();
    return e;
}

template <class G>
cudaError_t attr_geometry()
{
    cudaError_t e = attr_all<G, false, false>();
    if (e == cudaSuccess) e = attr_all<G, false, true>();
    if (e == cudaSuccess) e = attr_all<G, true, false>();
    if (e == cudaSuccess) e = attr_all<G, true, true>();
    return e;
}

template <class G, bool BG, bool HD>
cudaError_t launch_g(const BatchArgs& a, int stage, int grid, cudaStream_t s)
{
    const size_t sm = sizeof(f32k::Smem<G>);
    switch (stage) {
        case 1: stage_fp32_batch<G, 1, BG, HD><<<grid, G::NT, sm, s>>>(a); break;
        case 2: stage_fp32_batch<G, 2, BG, HD><<<grid, G::NT, sm, s>>>(a); break;
        case 3: stage_fp32_batch<G, 3, BG, HD><<<grid, G::NT, sm, s>>>(a); break;
        default: stage_fp32_batch<G, 4, BG, HD><<<grid, G::NT, sm, s>>>(a); break;
    }
    return cudaGetLastError();
}

template <bool BG, bool HD>
cudaError_t launch(const BatchArgs& a, int tile, int stage, int grid, cudaStream_t s)
{
    switch (tile) {
        case TILE_64x16: return launch_g<f32k::G64x16, BG, HD>(a, stage, grid, s);
        case TILE_32x16: return launch_g<f32k::G32x16, BG, HD>(a, stage, grid, s);
        default: return launch_g<f32k::G32x32, BG, HD>(a, stage, grid, s);
    }
}

// (cells wide, cells high, resident CTAs per SM of the launch bounds) of a tile shape
void tile_dims(int tile, int& tx, int& ty, int& minb)
{
    if (tile == TILE_64x16) { tx = f32k::G64x16::TX; ty = f32k::G64x16::TY; minb = f32k::G64x16::MINB; }
    else if (tile == TILE_32x16) { tx = f32k::G32x16::TX; ty = f32k::G32x16::TY; minb = f32k::G32x16::MINB; }
    else { tx = f32k::G32x32::TX; ty = f32k::G32x32::TY; minb = f32k::G32x32::MINB; }
}

}  // namespace

struct sac_batch {
    int n = 0;
    std::vector<sac_ctx*> runs;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    bool hd = true, bg = false;
    int nsm = 148;
    long long max_halo = 0;         // largest ghost frame over the runs (cells)
    bool any_halo = false;          // some run has a periodic or outflow boundary
    StageArgs<float>* d_args = nullptr;
    RunCtl* d_ctl = nullptr;
    int4* d_tiles = nullptr;
    unsigned* d_counters = nullptr;
    CUtensorMap* d_tmaps = nullptr;   // [n][4], or null (row copies)
    int ntiles = 0;
    int persistent = 1, ctas_per_sm = 2, order = 1, tile = TILE_32x32;
    std::vector<StageArgs<float>> h_args;   // host copy of d_args (re-encoded when the tile shape changes)
    cudaGraphExec_t g1 = nullptr, gN = nullptr;
    char err[512] = {0};
};

static int bfail(sac_batch* b, int code, const char* fmt, ...)
{
    if (b) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b->err, sizeof(b->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define BK(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? SAC_ERR_OOM : SAC_ERR_CUDA,  \
                         "%s failed: %s", #call, cudaGetErrorString(e_));                  \
    } while (0)

// Tile queue for one order:
//  0: runs in the given order, tiles row-major within a run;
//  1: runs by decreasing cell count (big runs first balance the tail);
//  2: runs by decreasing cell count, tiles interleaved round-robin across runs.
static std::vector<int4> make_tiles(const sac_batch* b, int order, int tile)
{
    int tw, th, minb;
    tile_dims(tile, tw, th, minb);
    std::vector<int> idx(b->n);
    for (int i = 0; i < b->n; ++i) idx[i] = i;
    if (order >= 1)
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) {
            return (long long)b->runs[a]->p.nx * b->runs[a]->p.ny > (long long)b->runs[c]->p.nx * b->runs[c]->p.ny;
        });
    std::vector<std::vector<int4>> per(b->n);
    for (int r : idx) {
        const int tx = (b->runs[r]->p.nx + tw - 1) / tw, ty = (b->runs[r]->p.ny + th - 1) / th;
        for (int y = 0; y < ty; ++y)
            for (int x = 0; x < tx; ++x) per[r].push_back(make_int4(r, x, y, 0));
    }
    std::vector<int4> out;
    if (order <= 1) {
        for (int r : idx) out.insert(out.end(), per[r].begin(), per[r].end());
    } else {
        size_t most = 0;
        for (int r : idx) most = std::max(most, per[r].size());
        for (size_t k = 0; k < most; ++k)
            for (int r : idx)
                if (k < per[r].size()) out.push_back(per[r][k]);
    }
    return out;
}

static cudaError_t enqueue_batch_step(sac_batch* b, cudaStream_t s)
{
    batch_begin_kernel<<<(b->n + 127) / 128, 128, 0, s>>>(b->d_ctl, b->n, b->d_counters);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    BatchArgs a;
    a.args = b->d_args; a.tiles = b->d_tiles; a.ntiles = b->ntiles; a.counters = b->d_counters;
    a.tmaps = b->d_tmaps;
    a.persistent = b->persistent;
    int tw, th, minb;
    tile_dims(b->tile, tw, th, minb);
    // ctas_per_sm 2: as many CTAs per SM as the tile shape's launch bounds allow
    const int per_sm = b->ctas_per_sm == 1 ? 1 : minb;
    const int grid = b->persistent ? std::min(b->ntiles, per_sm * b->nsm) : b->ntiles;
    const int hgrid = (int)std::min<long long>((b->max_halo + 255) / 256, 2 * b->nsm);
    const int T = b->tile;
    for (int stage = 1; stage <= 4 && e == cudaSuccess; ++stage) {
        if (b->bg) e = b->hd ? launch<true, true>(a, T, stage, grid, s) : launch<true, false>(a, T, stage, grid, s);
        else e = b->hd ? launch<false, true>(a, T, stage, grid, s) : launch<false, false>(a, T, stage, grid, s);
        if (e == cudaSuccess && b->any_halo) {
            halo_fp32_batch<<<dim3(hgrid, b->n), 256, 0, s>>>(b->d_args, stage);
            e = cudaGetLastError();
        }
    }
    return e;
}

static void drop_graphs(sac_batch* b)
{
    if (b->g1) cudaGraphExecDestroy(b->g1);
    if (b->gN) cudaGraphExecDestroy(b->gN);
    b->g1 = b->gN = nullptr;
}

static cudaError_t capture_batch(sac_batch* b, int nsteps, cudaGraphExec_t* out)
{
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k) e = enqueue_batch_step(b, b->cap);
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

// Upload the run arguments and tensor maps for tile shape `tile` (the tensor
// maps' boxes follow the shape); without tensor maps the kernel copies rows.
static int set_tile_tables(sac_batch* b, int tile)
{
    for (auto& a : b->h_args) { a.tile = tile; a.kernel_ghosts = 0; }
    BK(cudaMemcpy(b->d_args, b->h_args.data(), b->h_args.size() * sizeof(StageArgs<float>), cudaMemcpyHostToDevice));
    if (b->d_tmaps) {
        std::vector<CUtensorMap> maps(b->h_args.size());
        bool ok = true;
        for (size_t k = 0; k < maps.size() && ok; ++k) ok = encode_stage_tensor_map(b->h_args[k], &maps[k]) == cudaSuccess;
        if (!ok || cudaMemcpy(b->d_tmaps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(b->d_tmaps);
            b->d_tmaps = nullptr;
        }
    }
    return SAC_OK;
}

static int apply_config(sac_batch* b, int persistent, int ctas, int order, int tile)
{
    if (persistent < 0 || persistent > 2 || ctas < 1 || ctas > 2 || order < 0 || order > 2 || tile < 0 ||
        tile >= NTILE_SHAPES)
        return bfail(b, SAC_ERR_ARG, "bad configuration (%d, %d, %d, %d)", persistent, ctas, order, tile);
    BK(cudaStreamSynchronize(b->stream));
    if (tile != b->tile) {
        int rc = set_tile_tables(b, tile);
        if (rc != SAC_OK) return rc;
        b->tile = tile;
    }
    std::vector<int4> t = make_tiles(b, order, tile);
    BK(cudaMemcpyAsync(b->d_tiles, t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream));
    BK(cudaStreamSynchronize(b->stream));
    b->ntiles = (int)t.size();
    b->persistent = persistent; b->ctas_per_sm = ctas; b->order = order;
    drop_graphs(b);
    return SAC_OK;
}

extern "C" {

const char* sac_batch_last_error(const sac_batch* b) { return b ? b->err : "no batch"; }

void sac_batch_free(sac_batch* b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    for (sac_ctx* c : b->runs) sac_free(c);
    cudaFree(b->d_args); cudaFree(b->d_ctl); cudaFree(b->d_tiles); cudaFree(b->d_counters); cudaFree(b->d_tmaps);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

int sac_batch_init(const sac_params* runs, int n, sac_batch** out)
{
    if (out) *out = nullptr;
    if (!runs || !out || n < 1 || n > 65535) return SAC_ERR_ARG;   // one halo grid row per run
    for (int i = 0; i < n; ++i) {
        if (runs[i].precision != SAC_FP32 || runs[i].device != runs[0].device || runs[i].stream != runs[0].stream ||
            runs[i].hyperdiffusion != runs[0].hyperdiffusion || runs[i].has_background != runs[0].has_background ||
            runs[i].gravity[0] != 0.0 || runs[i].gravity[1] != 0.0 || runs[i].hd_single_face)
            return SAC_ERR_ARG;
    }
    sac_batch* b = new sac_batch();
    b->n = n;
    b->stream = (cudaStream_t)runs[0].stream;
    b->hd = runs[0].hyperdiffusion != 0;
    b->bg = runs[0].has_background != 0;
    for (int i = 0; i < n; ++i) {
        sac_ctx* c = nullptr;
        int rc = sac_init(&runs[i], &c);
        if (rc != SAC_OK) {
            bfail(b, rc, "run %d: sac_init failed (%s)", i, sac_status_string(rc));
            sac_batch_free(b);
            return rc;
        }
        b->runs.push_back(c);
    }
    int rc = SAC_OK;
    do {
        cudaError_t e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, runs[0].device);
        if (e == cudaSuccess) e = attr_geometry<f32k::G32x32>();
        if (e == cudaSuccess) e = attr_geometry<f32k::G64x16>();
        if (e == cudaSuccess) e = attr_geometry<f32k::G32x16>();
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) { rc = bfail(b, SAC_ERR_CUDA, "set-up: %s", cudaGetErrorString(e)); break; }
        std::vector<StageArgs<float>> args(4 * n);
        std::vector<RunCtl> ctl(n);
        long long ntiles = 0;   // the most tiles any shape needs (the table holds any shape's queue)
        for (int i = 0; i < n; ++i) {
            const sac_ctx* c = b->runs[i];
            for (int s = 1; s <= 4; ++s) sac_fp32_stage_args(c, s, &args[4 * i + s - 1]);
            if (c->p.bc_x != BC_FIXED || c->p.bc_y != BC_FIXED) {
                b->any_halo = true;
                b->max_halo = std::max(b->max_halo, f32k::halo_count(c->L));
            }
            ctl[i].sc = c->sc;
            ctl[i].dx = c->dx;
            ctl[i].dy = c->dy;
            ctl[i].courant = c->p.courant;
            long long most = 0;
            for (int t = 0; t < NTILE_SHAPES; ++t) {
                int tw, th, minb;
                tile_dims(t, tw, th, minb);
                most = std::max(most, (long long)((c->p.nx + tw - 1) / tw) * ((c->p.ny + th - 1) / th));
            }
            ntiles += most;
        }
        if (ntiles > (1LL << 30)) { rc = bfail(b, SAC_ERR_ARG, "too many tiles"); break; }
        b->ntiles = (int)ntiles;
        if (cudaMalloc(&b->d_args, args.size() * sizeof(StageArgs<float>)) != cudaSuccess ||
            cudaMalloc(&b->d_ctl, n * sizeof(RunCtl)) != cudaSuccess ||
            cudaMalloc(&b->d_tiles, ntiles * sizeof(int4)) != cudaSuccess ||
            cudaMalloc(&b->d_counters, 4 * sizeof(unsigned)) != cudaSuccess) {
            rc = bfail(b, SAC_ERR_OOM, "batch tables");
            break;
        }
        e = cudaMemcpy(b->d_args, args.data(), args.size() * sizeof(StageArgs<float>), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->d_ctl, ctl.data(), n * sizeof(RunCtl), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(b->d_counters, 0, 4 * sizeof(unsigned));
        if (e != cudaSuccess) { rc = bfail(b, SAC_ERR_CUDA, "tables: %s", cudaGetErrorString(e)); break; }
        b->h_args = args;
        if (cudaMalloc(&b->d_tmaps, args.size() * sizeof(CUtensorMap)) != cudaSuccess) {
            cudaGetLastError();
            b->d_tmaps = nullptr;
        }
        if ((rc = set_tile_tables(b, TILE_32x32)) != SAC_OK) break;
        rc = apply_config(b, 1, 2, 1, TILE_32x32);
    } while (0);
    if (rc != SAC_OK) {
        sac_batch_free(b);
        return rc;
    }
    *out = b;
    return SAC_OK;
}

int sac_batch_set_state(sac_batch* b, int run, const double* w, const double* bg, double t)
{
    if (!b || run < 0 || run >= b->n) return bfail(b, SAC_ERR_ARG, "bad run index");
    int rc = sac_set_state(b->runs[run], w, bg, t);
    if (rc != SAC_OK) return bfail(b, rc, "run %d: %s", run, sac_last_error(b->runs[run]));
    return SAC_OK;
}

int sac_batch_get_state(sac_batch* b, int run, double* w, double* t)
{
    if (!b || run < 0 || run >= b->n) return bfail(b, SAC_ERR_ARG, "bad run index");
    int rc = sac_get_state(b->runs[run], w, t);
    if (rc != SAC_OK) return bfail(b, rc, "run %d: %s", run, sac_last_error(b->runs[run]));
    return SAC_OK;
}

int sac_batch_time(sac_batch* b, int run, double* t, long* steps)
{
    if (!b || run < 0 || run >= b->n) return bfail(b, SAC_ERR_ARG, "bad run index");
    int rc = sac_time(b->runs[run], t, steps);
    if (rc != SAC_OK) return bfail(b, rc, "run %d: %s", run, sac_last_error(b->runs[run]));
    return SAC_OK;
}

int sac_batch_steps(sac_batch* b, long nsteps)
{
    if (!b) return SAC_ERR_ARG;
    if (nsteps < 0) return bfail(b, SAC_ERR_ARG, "nsteps < 0");
    for (int i = 0; i < b->n; ++i)
        if (!b->runs[i]->have_state) return bfail(b, SAC_ERR_STATE, "run %d has no state", i);
    // both step graphs are captured by the first call (a one-time set-up)
    if (!b->g1) BK(capture_batch(b, 1, &b->g1));
    if (!b->gN) BK(capture_batch(b, kChunk, &b->gN));
    long left = nsteps;
    while (left >= kChunk) { BK(cudaGraphLaunch(b->gN, b->stream)); left -= kChunk; }
    while (left > 0) { BK(cudaGraphLaunch(b->g1, b->stream)); --left; }
    return SAC_OK;
}

int sac_batch_sync(sac_batch* b)
{
    if (!b) return SAC_ERR_ARG;
    BK(cudaStreamSynchronize(b->stream));
    for (int i = 0; i < b->n; ++i) {
        int rc = sac_sync(b->runs[i]);
        if (rc != SAC_OK) return bfail(b, rc, "run %d: %s", i, sac_last_error(b->runs[i]));
    }
    return SAC_OK;
}

int sac_batch_set_config(sac_batch* b, int persistent, int ctas_per_sm, int order)
{
    if (!b) return SAC_ERR_ARG;
    return apply_config(b, persistent, ctas_per_sm, order, b->tile);
}

int sac_batch_set_tile(sac_batch* b, int tile)
{
    if (!b) return SAC_ERR_ARG;
    return apply_config(b, b->persistent, b->ctas_per_sm, b->order, tile);
}

int sac_batch_get_config(const sac_batch* b, int config[4])
{
    if (!b || !config) return SAC_ERR_ARG;
    config[0] = b->persistent; config[1] = b->ctas_per_sm; config[2] = b->order; config[3] = b->tile;
    return SAC_OK;
}

int sac_batch_tune(sac_batch* b, int trials, int config[3], double* ms_out)
{
    if (!b) return SAC_ERR_ARG;
    if (trials < 1) return bfail(b, SAC_ERR_ARG, "trials < 1");
    for (int i = 0; i < b->n; ++i)
        if (!b->runs[i]->have_state) return bfail(b, SAC_ERR_STATE, "run %d has no state", i);
    // snapshot every run's state and scalars; trials advance them
    std::vector<void*> snap(b->n, nullptr);
    std::vector<DevScalars> ssc(b->n);
    int rc = SAC_OK;
    for (int i = 0; i < b->n && rc == SAC_OK; ++i) {
        sac_ctx* c = b->runs[i];
        const size_t bytes = NF * (size_t)c->L.fstride * c->esz;
        if (cudaMalloc(&snap[i], bytes) != cudaSuccess) { rc = bfail(b, SAC_ERR_OOM, "tuner snapshot"); break; }
        if (cudaMemcpyAsync(snap[i], c->u0, bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess ||
            cudaMemcpyAsync(&ssc[i], c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
            rc = bfail(b, SAC_ERR_CUDA, "tuner snapshot copy");
    }
    if (rc == SAC_OK && cudaStreamSynchronize(b->stream) != cudaSuccess) rc = bfail(b, SAC_ERR_CUDA, "sync");
    const int cfg[][3] = {{1, 2, 0}, {1, 2, 1}, {1, 2, 2}, {1, 1, 0}, {1, 1, 1}, {1, 1, 2},
                          {0, 2, 0}, {0, 2, 1}, {0, 2, 2}, {2, 2, 0}, {2, 2, 1}, {2, 2, 2}};
    const int ncfg = (int)(sizeof cfg / sizeof cfg[0]);
    std::vector<std::array<int, 4>> cand;
    for (int t = 0; t < NTILE_SHAPES; ++t)
        for (int k = 0; k < ncfg; ++k) cand.push_back({cfg[k][0], cfg[k][1], cfg[k][2], t});
    const int ncand = (int)cand.size();
    double best = 1e300;
    int bi = 1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == SAC_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = bfail(b, SAC_ERR_CUDA, "events");
    for (int k = 0; k < ncand && rc == SAC_OK; ++k) {
        if ((rc = apply_config(b, cand[k][0], cand[k][1], cand[k][2], cand[k][3])) != SAC_OK) break;
        if (enqueue_batch_step(b, b->stream) != cudaSuccess) { rc = bfail(b, SAC_ERR_CUDA, "trial"); break; }
        cudaEventRecord(e0, b->stream);
        for (int t = 0; t < trials; ++t)
            if (enqueue_batch_step(b, b->stream) != cudaSuccess) { rc = bfail(b, SAC_ERR_CUDA, "trial"); break; }
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = bfail(b, SAC_ERR_CUDA, "trial sync"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms / trials < best) { best = ms / trials; bi = k; }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    // restore states and scalars
    for (int i = 0; i < b->n; ++i) {
        sac_ctx* c = b->runs[i];
        if (snap[i]) {
            const size_t bytes = NF * (size_t)c->L.fstride * c->esz;
            cudaMemcpyAsync(c->u0, snap[i], bytes, cudaMemcpyDeviceToDevice, b->stream);
            cudaMemcpyAsync(c->sc, &ssc[i], sizeof(DevScalars), cudaMemcpyHostToDevice, b->stream);
        }
    }
    cudaStreamSynchronize(b->stream);
    for (void* p : snap) cudaFree(p);
    if (rc != SAC_OK) return rc;
    rc = apply_config(b, cand[bi][0], cand[bi][1], cand[bi][2], cand[bi][3]);
    if (rc != SAC_OK) return rc;
    if (config) { config[0] = cand[bi][0]; config[1] = cand[bi][1]; config[2] = cand[bi][2]; }
    if (ms_out) *ms_out = best;
    return SAC_OK;
}

}  // extern "C"
