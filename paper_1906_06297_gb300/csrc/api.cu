// api.cu -- the C ABI of libising (declared in include/ising.h): argument
// checks, the FP64 acceptance table, and the launch sequence of a sweep.
//
// Every entry point validates its arguments before queueing work and returns
// a status; device planes are checked to be device memory of the current
// device that covers the whole plane (cuMemGetAddressRange through the
// runtime's driver entry point), so a wrong size or a host pointer becomes
// ISING_EINVAL instead of an out-of-bounds access on the GPU.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/ising.h"
#include "common.cuh"
#include "launch.h"

namespace ising {

namespace {

thread_local char g_last_error[256] = "";


int fail(int status, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return status;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(ISING_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

struct DeviceCache {
    std::mutex mu;
    std::mutex host_mu;  // held while ising_sweep_host enqueues its bands
    int sm_count[64] = {};
    cudaStream_t aux[64][3] = {};  // compute, copy-out and capture streams of ising_sweep_host, made on first use
    cudaGraphExec_t host_exec[64] = {};  // the last banded schedule, replayed (updated) by the next call
    cudaEvent_t *host_ev[64] = {};  // the events of ising_sweep_host's bands, made on first use
};
DeviceCache g_dev;

int row_bytes_of(int64_t L, int32_t layout, size_t *row)
{
    if (L <= 0 || (L & 1)) return fail(ISING_EINVAL, "L = %lld must be positive and even", (long long)L);
    if (L > (int64_t(1) << 31)) return fail(ISING_EINVAL, "L = %lld is too large", (long long)L);
    if (layout == ISING_INT8) {
        *row = (size_t)(L / 2);
    } else if (layout == ISING_MSC4) {
        if (L % 64 != 0) return fail(ISING_EINVAL, "MSC4 needs L %% 64 == 0 (L = %lld)", (long long)L);
        *row = (size_t)(L / 32) * sizeof(uint64_t);
    } else {
        return fail(ISING_EINVAL, "unknown layout %d", (int)layout);
    }
    return ISING_OK;
}

int check_lattice(const ising_lattice_t *lat)
{
    if (lat == nullptr) return fail(ISING_EINVAL, "lattice is NULL");
    size_t row = 0;
    int rc = row_bytes_of(lat->L, lat->layout, &row);
    if (rc) return rc;
    if (lat->reserved != 0) return fail(ISING_EINVAL, "reserved field must be 0");
    if (lat->row_stride_bytes < (int64_t)row)
        return fail(ISING_EINVAL, "row stride %lld < row size %zu", (long long)lat->row_stride_bytes, row);
    if (lat->black == lat->white) return fail(ISING_EINVAL, "black and white planes alias");
    if (lat->layout == ISING_MSC4) {
        if (lat->row_stride_bytes % 16 != 0) return fail(ISING_EINVAL, "MSC4 row stride must be a multiple of 16");
        if (((uintptr_t)lat->black | (uintptr_t)lat->white) % 16 != 0)
            return fail(ISING_EINVAL, "MSC4 planes must be 16-byte aligned");
    }
    const size_t plane = (size_t)(lat->L - 1) * (size_t)lat->row_stride_bytes + row;
    const char *b = (const char *)lat->black, *w = (const char *)lat->white;
    if ((b < w && b + plane > w) || (w < b && w + plane > b)) return fail(ISING_EINVAL, "planes overlap");
    rc = check_device_range(lat->black, plane, "black plane");
    if (rc) return rc;
    return check_device_range(lat->white, plane, "white plane");
}

int build_accept(double beta, Accept *acc, uint64_t T[5])
{
    int rc = ising_thresholds(beta, T);
    if (rc) return rc;
    const uint64_t two32 = uint64_t(1) << 32;
    if (T[0] != two32 || T[1] != two32 || T[2] != two32)
        return fail(ISING_EINVAL, "beta = %g gives a non-trivial threshold for dE <= 0", beta);
    acc->T3_64 = T[3];
    acc->T4_64 = T[4];
    // T4 <= T3 for beta >= 0, and T3 reaches 2^32 only at beta = 0, where T4
    // does too; the kernels then mask out the threshold test entirely
    if (T[4] > T[3] || (T[3] >= two32) != (T[4] >= two32))
        return fail(ISING_EINVAL, "beta = %g gives an unordered threshold table", beta);
    acc->always = T[3] >= two32 ? 1u : 0u;
    acc->zero = 0u;
    acc->T3 = T[3] >= two32 ? 0xffffffffu : (uint32_t)T[3];
    acc->T4 = T[4] >= two32 ? 0xffffffffu : (uint32_t)T[4];
    return ISING_OK;
}

int half_sweep_impl(const ising_lattice_t *lat, const Accept &acc, const RoundKeys &rk, int colour, uint64_t t,
                    int64_t *obs, cudaStream_t s)
{
    const uint32_t c2 = (uint32_t)t, c3 = counter_word3(colour, kPurposeMetropolis, t);
    cudaError_t e;
    if (lat->layout == ISING_MSC4) {
        Msc4SweepParams p;
        p.tgt = (uint64_t *)(colour == 0 ? lat->black : lat->white);
        p.src = (const uint64_t *)(colour == 0 ? lat->white : lat->black);
        p.L = lat->L;
        p.rows = lat->L;
        p.row0 = 0;
        p.wrap_row = lat->L;  // periodic: row L is row 0
        p.wrap_to = 0;
        p.first_up = lat->L - 1;
        p.wpr = lat->L / 32;
        p.stride = lat->row_stride_bytes / 8;
        p.qrow = lat->L / 8;
        p.total = ((p.wpr + 63) / 64) * lat->L;
        p.c2 = c2;
        p.c3 = c3;
        p.acc = acc;
        p.rk = rk;
        p.obs = (long long *)obs;
        e = msc4_half_sweep(p, colour, s);
    } else {
        Int8SweepParams p;
        p.tgt = (int8_t *)(colour == 0 ? lat->black : lat->white);
        p.src = (const int8_t *)(colour == 0 ? lat->white : lat->black);
        p.L = lat->L;
        p.half = lat->L / 2;
        p.stride = lat->row_stride_bytes;
        p.nblk = (lat->L * (lat->L / 2) + 3) / 4;
        p.c2 = c2;
        p.c3 = c3;
        p.acc = acc;
        p.rk = rk;
        p.obs = (long long *)obs;
        e = int8_half_sweep(p, colour, s);
    }
    return e == cudaSuccess ? ISING_OK : cuda_fail(e, "half-sweep launch");
}

constexpr int kMaxSlabs = kMaxHaloRows / 2;

size_t slab_plane_bytes(const ising_slab_t *sl)
{
    return (size_t)(sl->rows + 1) * (size_t)sl->row_stride_bytes + (size_t)(sl->L / 4);
}

int check_slab(const ising_slab_t *sl)
{
    if (sl == nullptr) return fail(ISING_EINVAL, "slab is NULL");
    if (sl->layout != ISING_MSC4) return fail(ISING_EINVAL, "slabs support the MSC4 layout only");
    size_t row = 0;
    int rc = row_bytes_of(sl->L, sl->layout, &row);
    if (rc) return rc;
    if (sl->spare_sms < 0 || sl->spare_sms > 4095) return fail(ISING_EINVAL, "spare_sms = %d out of range", sl->spare_sms);
    if (sl->rows < 1) return fail(ISING_EINVAL, "slab rows = %lld must be >= 1", (long long)sl->rows);
    if (sl->row0 < 0 || sl->row0 >= sl->L || sl->rows > sl->L - sl->row0)
        return fail(ISING_EINVAL, "slab rows [%lld, %lld) are not inside 0..L-1 (L = %lld)", (long long)sl->row0,
                    (long long)(sl->row0 + sl->rows), (long long)sl->L);
    if (sl->row_stride_bytes < (int64_t)row)
        return fail(ISING_EINVAL, "row stride %lld < row size %zu", (long long)sl->row_stride_bytes, row);
    if (sl->row_stride_bytes % 16 != 0) return fail(ISING_EINVAL, "MSC4 row stride must be a multiple of 16");
    if (((uintptr_t)sl->black | (uintptr_t)sl->white) % 16 != 0)
        return fail(ISING_EINVAL, "MSC4 planes must be 16-byte aligned");
    const size_t plane = slab_plane_bytes(sl);
    const char *b = (const char *)sl->black, *w = (const char *)sl->white;
    if (b == w || (b < w && b + plane > w) || (w < b && w + plane > b)) return fail(ISING_EINVAL, "planes overlap");
    rc = check_device_range(sl->black, plane, "black slab plane");
    if (rc) return rc;
    return check_device_range(sl->white, plane, "white slab plane");
}

// n slabs that tile the rows of one lattice in order, with no plane shared.
int check_slab_set(const ising_slab_t *slabs, int32_t n)
{
    if (slabs == nullptr) return fail(ISING_EINVAL, "slabs is NULL");
    if (n < 1 || n > kMaxSlabs) return fail(ISING_EINVAL, "n = %d slabs, must be 1..%d", (int)n, kMaxSlabs);
    int64_t next = 0;
    for (int32_t k = 0; k < n; ++k) {
        int rc = check_slab(&slabs[k]);
        if (rc) return rc;
        if (slabs[k].L != slabs[0].L) return fail(ISING_EINVAL, "slab %d has another L", (int)k);
        if (slabs[k].row0 != next)
            return fail(ISING_EINVAL, "slab %d starts at row %lld, expected %lld", (int)k, (long long)slabs[k].row0,
                        (long long)next);
        next += slabs[k].rows;
    }
    if (next != slabs[0].L)
        return fail(ISING_EINVAL, "slabs cover rows 0..%lld, not the lattice's %lld", (long long)next - 1,
                    (long long)slabs[0].L);
    for (int32_t a = 0; a < n; ++a)
        for (int32_t b = a + 1; b < n; ++b) {
            const char *pa[2] = {(const char *)slabs[a].black, (const char *)slabs[a].white};
            const char *pb[2] = {(const char *)slabs[b].black, (const char *)slabs[b].white};
            const size_t na = slab_plane_bytes(&slabs[a]), nb = slab_plane_bytes(&slabs[b]);
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j)
                    if (pa[i] < pb[j] + nb && pb[j] < pa[i] + na)
                        return fail(ISING_EINVAL, "planes of slabs %d and %d overlap", (int)a, (int)b);
        }
    return ISING_OK;
}

// Half-sweep of rows row0 .. row0 + rows - 1 of a periodic MSC4 lattice, in
// place: local row r is global row row0 + r; the source walk reaches global
// rows row0 - 1 .. row0 + rows + 1 (mod L), so the row above local row 0 is
// local L - 1 for the first band and local -1 otherwise, and global row L
// (local L - row0) continues at global row 0 (local -row0).  Keys, thresholds
// and observables are those of the whole-lattice half-sweep restricted to the
// band, so the bands of a partition give the whole-lattice result bit for bit.
int band_half_sweep_impl(const ising_lattice_t *lat, const Accept &acc, const RoundKeys &rk, int colour, uint64_t t,
                         int64_t row0, int64_t rows, int64_t *obs, cudaStream_t s)
{
    const int64_t stride = lat->row_stride_bytes / 8;
    Msc4SweepParams p;
    p.tgt = (uint64_t *)(colour == 0 ? lat->black : lat->white) + row0 * stride;
    p.src = (const uint64_t *)(colour == 0 ? lat->white : lat->black) + row0 * stride;
    p.L = lat->L;
    p.rows = rows;
    p.row0 = row0;
    p.wrap_row = lat->L - row0;
    p.wrap_to = -row0;
    p.first_up = row0 == 0 ? lat->L - 1 : -1;
    p.wpr = lat->L / 32;
    p.stride = stride;
    p.qrow = lat->L / 8;
    p.total = ((p.wpr + 63) / 64) * rows;
    p.c2 = (uint32_t)t;
    p.c3 = counter_word3(colour, kPurposeMetropolis, t);
    p.acc = acc;
    p.rk = rk;
    p.obs = (long long *)obs;
    cudaError_t e = msc4_half_sweep(p, colour, s);
    return e == cudaSuccess ? ISING_OK : cuda_fail(e, "band half-sweep launch");
}

// The compute and copy-out streams of the banded host path, per device.
int aux_streams(cudaStream_t *cmp, cudaStream_t *out, cudaStream_t *cap = nullptr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(ISING_ECUDA, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_dev.mu);
    for (int i = 0; i < 3; ++i)
        if (g_dev.aux[dev][i] == nullptr) {
            e = cudaStreamCreateWithFlags(&g_dev.aux[dev][i], cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(e, "stream create");
        }
    *cmp = g_dev.aux[dev][0];
    *out = g_dev.aux[dev][1];
    if (cap) *cap = g_dev.aux[dev][2];
    return ISING_OK;
}

int slab_half_sweep_impl(const ising_slab_t *sl, const Accept &acc, const RoundKeys &rk, int colour, uint64_t t,
                         int64_t *obs, cudaStream_t s)
{
    const int64_t stride = sl->row_stride_bytes / 8;
    Msc4SweepParams p;
    // local row 0 = plane row 1; the halos are local rows -1 and `rows`
    p.tgt = (uint64_t *)(colour == 0 ? sl->black : sl->white) + stride;
    p.src = (const uint64_t *)(colour == 0 ? sl->white : sl->black) + stride;
    p.L = sl->L;
    p.rows = sl->rows;
    p.row0 = sl->row0;
    p.wrap_row = sl->rows + 1;  // only the prefetch after the last row gets there
    p.wrap_to = -1;
    p.first_up = -1;
    p.wpr = sl->L / 32;
    p.stride = stride;
    p.qrow = sl->L / 8;
    p.total = ((p.wpr + 63) / 64) * sl->rows;
    p.c2 = (uint32_t)t;
    p.c3 = counter_word3(colour, kPurposeMetropolis, t);
    p.acc = acc;
    p.rk = rk;
    p.obs = (long long *)obs;
    p.spare_sms = sl->spare_sms;
    DeviceInfo info;
    cudaError_t e = device_info(&info);
    if (e != cudaSuccess) return cuda_fail(e, "device info");
    if (sl->spare_sms >= info.sm_count)
        return fail(ISING_EINVAL, "spare_sms = %d leaves no SM of %d", sl->spare_sms, info.sm_count);
    e = msc4_half_sweep(p, colour, s);
    return e == cudaSuccess ? ISING_OK : cuda_fail(e, "slab half-sweep launch");
}

int slab_exchange_impl(const ising_slab_t *slabs, int32_t n, int colour, cudaStream_t s)
{
    HaloCopy c;
    for (int32_t k = 0; k < n; ++k) {
        const ising_slab_t &me = slabs[k], &up = slabs[(k + n - 1) % n], &dn = slabs[(k + 1) % n];
        auto row = [colour](const ising_slab_t &sl, int64_t r) {
            return (uint64_t *)((char *)(colour == 0 ? sl.black : sl.white) + r * sl.row_stride_bytes);
        };
        c.src[2 * k] = row(up, up.rows);  // last own row of the slab above
        c.dst[2 * k] = row(me, 0);
        c.src[2 * k + 1] = row(dn, 1);  // first own row of the slab below
        c.dst[2 * k + 1] = row(me, me.rows + 1);
    }
    cudaError_t e = msc4_copy_rows(c, 2 * n, slabs[0].L / 32, s);
    return e == cudaSuccess ? ISING_OK : cuda_fail(e, "halo copy launch");
}

}  // namespace

typedef CUresult (*AddressRangeFn)(CUdeviceptr *base, size_t *size, CUdeviceptr ptr);

AddressRangeFn address_range_fn()
{
    static AddressRangeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<AddressRangeFn>(p);
    });
    return fn;
}

// ptr must be device (or managed) memory usable by the current device, with
// [ptr, ptr + bytes) inside one allocation.
int check_device_range(const void *ptr, size_t bytes, const char *name)
{
    if (ptr == nullptr) return fail(ISING_EINVAL, "%s is NULL", name);
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ISING_EINVAL, "%s is not a CUDA pointer (%s)", name, cudaGetErrorString(e));
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(ISING_EINVAL, "%s is not device memory", name);
    int dev = -1;
    cudaGetDevice(&dev);
    if (at.type == cudaMemoryTypeDevice && at.device != dev)
        return fail(ISING_EINVAL, "%s lives on device %d, current device is %d", name, at.device, dev);
    AddressRangeFn fn = address_range_fn();
    if (fn != nullptr) {
        CUdeviceptr base = 0;
        size_t size = 0;
        if (fn(&base, &size, (CUdeviceptr)ptr) == CUDA_SUCCESS) {
            const size_t off = (size_t)((CUdeviceptr)ptr - base);
            if (off > size || size - off < bytes)
                return fail(ISING_EINVAL, "%s: %zu bytes needed, allocation has %zu past the pointer", name, bytes,
                            size - off);
        }
    }
    return ISING_OK;
}


cudaError_t device_info(DeviceInfo *info)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_dev.mu);
    if (g_dev.sm_count[dev] == 0) {
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_dev.sm_count[dev] = n;
    }
    info->sm_count = g_dev.sm_count[dev];
    return cudaSuccess;
}

}  // namespace ising

using namespace ising;

extern "C" {

ISING_API const char *ising_strerror(int status)
{
    switch (status) {
    case ISING_OK: return "ok";
    case ISING_EINVAL: return "invalid argument";
    case ISING_ECUDA: return "CUDA error";
    case ISING_ETIMEOUT: return "device wait timed out";
    default: return "unknown status";
    }
}

ISING_API const char *ising_last_error(void) { return g_last_error; }

ISING_API int ising_lattice_bytes(int64_t L, int32_t layout, size_t *row_bytes, size_t *plane_bytes)
{
    size_t row = 0;
    int rc = row_bytes_of(L, layout, &row);
    if (rc) return rc;
    if (row_bytes) *row_bytes = row;
    if (plane_bytes) *plane_bytes = row * (size_t)L;
    return ISING_OK;
}

ISING_API int ising_thresholds(double beta, uint64_t T[5])
{
    if (T == nullptr) return fail(ISING_EINVAL, "T is NULL");
    if (!std::isfinite(beta) || beta < 0.0) return fail(ISING_EINVAL, "beta = %g must be finite and >= 0", beta);
    for (int a = 0; a <= 4; ++a) {
        // a aligned neighbours: flipping changes the energy by 2 s sum(nn) = 4a - 8
        const double p = std::exp(-beta * (4.0 * a - 8.0));
        T[a] = p >= 1.0 ? (uint64_t(1) << 32) : (uint64_t)std::floor(std::ldexp(p, 32));
    }
    return ISING_OK;
}

ISING_API int ising_init_lattice(const ising_lattice_t *lat, int32_t init, uint64_t seed, ising_stream_t stream)
{
    int rc = check_lattice(lat);
    if (rc) return rc;
    if (init < ISING_INIT_RANDOM || init > ISING_INIT_DOWN) return fail(ISING_EINVAL, "unknown init mode %d", init);
    cudaStream_t s = (cudaStream_t)stream;
    for (int colour = 0; colour < 2; ++colour) {
        void *plane = colour == 0 ? lat->black : lat->white;
        cudaError_t e = lat->layout == ISING_MSC4
                            ? msc4_init((uint64_t *)plane, colour, lat->L, lat->L, 0, lat->row_stride_bytes / 8,
                                        init, seed, s)
                            : int8_init((int8_t *)plane, colour, lat->L, lat->row_stride_bytes, init, seed, s);
        if (e != cudaSuccess) return cuda_fail(e, "init launch");
    }
    return ISING_OK;
}

ISING_API int ising_half_sweep(const ising_lattice_t *lat, double beta, int32_t colour, uint64_t seed, uint64_t t,
                               int64_t *obs_dev, ising_stream_t stream)
{
    int rc = check_lattice(lat);
    if (rc) return rc;
    if (colour != 0 && colour != 1) return fail(ISING_EINVAL, "colour must be 0 or 1");
    if (obs_dev != nullptr) {
        if (colour != 1) return fail(ISING_EINVAL, "observables are fused into the white half-sweep only");
        rc = check_device_range(obs_dev, 2 * sizeof(int64_t), "obs");
        if (rc) return rc;
    }
    Accept acc;
    uint64_t T[5];
    rc = build_accept(beta, &acc, T);
    if (rc) return rc;
    return half_sweep_impl(lat, acc, make_round_keys(seed), colour, t, obs_dev, (cudaStream_t)stream);
}

ISING_API int ising_sweep(const ising_lattice_t *lat, double beta, int64_t n_sweeps, uint64_t seed,
                          uint64_t sweep_offset, int64_t *trace_dev, ising_stream_t stream)
{
    int rc = check_lattice(lat);
    if (rc) return rc;
    if (n_sweeps < 0) return fail(ISING_EINVAL, "n_sweeps = %lld < 0", (long long)n_sweeps);
    Accept acc;
    uint64_t T[5];
    rc = build_accept(beta, &acc, T);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (trace_dev != nullptr && n_sweeps > 0) {
        rc = check_device_range(trace_dev, (size_t)n_sweeps * 2 * sizeof(int64_t), "trace");
        if (rc) return rc;
        cudaError_t e = cudaMemsetAsync(trace_dev, 0, (size_t)n_sweeps * 2 * sizeof(int64_t), s);
        if (e != cudaSuccess) return cuda_fail(e, "trace memset");
    }
    const RoundKeys rk = make_round_keys(seed);
    for (int64_t k = 0; k < n_sweeps; ++k) {
        const uint64_t t = sweep_offset + (uint64_t)k;
        rc = half_sweep_impl(lat, acc, rk, 0, t, nullptr, s);
        if (rc) return rc;
        rc = half_sweep_impl(lat, acc, rk, 1, t, trace_dev ? trace_dev + 2 * k : nullptr, s);
        if (rc) return rc;
    }
    return ISING_OK;
}

ISING_API int ising_slab_bytes(int64_t L, int64_t rows, int32_t layout, size_t *row_bytes, size_t *plane_bytes)
{
    if (layout != ISING_MSC4) return fail(ISING_EINVAL, "slabs support the MSC4 layout only");
    size_t row = 0;
    int rc = row_bytes_of(L, layout, &row);
    if (rc) return rc;
    if (rows < 1 || rows > L) return fail(ISING_EINVAL, "slab rows = %lld must be in 1..L", (long long)rows);
    if (row_bytes) *row_bytes = row;
    if (plane_bytes) *plane_bytes = row * (size_t)(rows + 2);
    return ISING_OK;
}

ISING_API int ising_slab_init(const ising_slab_t *slab, int32_t init, uint64_t seed, ising_stream_t stream)
{
    int rc = check_slab(slab);
    if (rc) return rc;
    if (init < ISING_INIT_RANDOM || init > ISING_INIT_DOWN) return fail(ISING_EINVAL, "unknown init mode %d", init);
    const int64_t stride = slab->row_stride_bytes / 8;
    for (int colour = 0; colour < 2; ++colour) {
        uint64_t *own = (uint64_t *)(colour == 0 ? slab->black : slab->white) + stride;
        cudaError_t e = msc4_init(own, colour, slab->L, slab->rows, slab->row0, stride, init, seed,
                                  (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "slab init launch");
    }
    return ISING_OK;
}

ISING_API int ising_slab_half_sweep(const ising_slab_t *slab, double beta, int32_t colour, uint64_t seed,
                                    uint64_t t, int64_t *obs_dev, ising_stream_t stream)
{
    int rc = check_slab(slab);
    if (rc) return rc;
    if (colour != 0 && colour != 1) return fail(ISING_EINVAL, "colour must be 0 or 1");
    if (obs_dev != nullptr) {
        if (colour != 1) return fail(ISING_EINVAL, "observables are fused into the white half-sweep only");
        rc = check_device_range(obs_dev, 2 * sizeof(int64_t), "obs");
        if (rc) return rc;
    }
    Accept acc;
    uint64_t T[5];
    rc = build_accept(beta, &acc, T);
    if (rc) return rc;
    return slab_half_sweep_impl(slab, acc, make_round_keys(seed), colour, t, obs_dev, (cudaStream_t)stream);
}

ISING_API int ising_slab_exchange(const ising_slab_t *slabs, int32_t n, int32_t colour, ising_stream_t stream)
{
    int rc = check_slab_set(slabs, n);
    if (rc) return rc;
    if (colour != 0 && colour != 1) return fail(ISING_EINVAL, "colour must be 0 or 1");
    return slab_exchange_impl(slabs, n, colour, (cudaStream_t)stream);
}

ISING_API int ising_slab_sweep(const ising_slab_t *slabs, int32_t n, double beta, int64_t n_sweeps, uint64_t seed,
                               uint64_t sweep_offset, int64_t *trace_dev, ising_stream_t stream)
{
    int rc = check_slab_set(slabs, n);
    if (rc) return rc;
    if (n_sweeps < 0) return fail(ISING_EINVAL, "n_sweeps = %lld < 0", (long long)n_sweeps);
    Accept acc;
    uint64_t T[5];
    rc = build_accept(beta, &acc, T);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (trace_dev != nullptr && n_sweeps > 0) {
        rc = check_device_range(trace_dev, (size_t)n_sweeps * 2 * sizeof(int64_t), "trace");
        if (rc) return rc;
        cudaError_t e = cudaMemsetAsync(trace_dev, 0, (size_t)n_sweeps * 2 * sizeof(int64_t), s);
        if (e != cudaSuccess) return cuda_fail(e, "trace memset");
    }
    const RoundKeys rk = make_round_keys(seed);
    for (int64_t k = 0; k < n_sweeps; ++k) {
        const uint64_t t = sweep_offset + (uint64_t)k;
        for (int colour = 0; colour < 2; ++colour) {
            rc = slab_exchange_impl(slabs, n, 1 - colour, s);  // halos of the source colour
            if (rc) return rc;
            for (int32_t j = 0; j < n; ++j) {
                rc = slab_half_sweep_impl(&slabs[j], acc, rk, colour, t,
                                          colour == 1 && trace_dev ? trace_dev + 2 * k : nullptr, s);
                if (rc) return rc;
            }
        }
    }
    return ISING_OK;
}

namespace {

// One sweep of an MSC4 lattice held in host memory, in K row bands so that
// the copies overlap the half-sweeps and each other (the host link, not the
// sweep, bounds this path).  The compute stream runs black band 0, black 1,
// then black k before white k-1 for k = 2 .. K-1, then white K-1 and white 0:
// black band k reads the white rows next to it unchanged (white k-1 runs after
// black k, white 0 last because black K-1 reads white row 0) and white band k
// needs black bands k-1 .. k+1 done.  Stream `s` copies plane bands in the
// order black bands first need them (white K-1, 0, 1, black 0, then white k+1
// and black k), so black k waits only for the copy of its own black band; the
// copy-out stream returns each plane band in compute order as soon as it is
// final -- a black band right after its black half-sweep -- so that both link
// directions stay busy from the first band to the last.  `s` finally waits for
// the copy-out stream.
//
// Host formats: with stage == nullptr the host planes are MSC4 rows of `hrow`
// bytes copied straight into the lattice; otherwise they are bit-packed rows
// of `hrow` = L/16 bytes, copied into `stage` (black's plane, then white's)
// and converted to and from MSC4 on the compute stream around each band's
// half-sweeps.
constexpr int kMaxHostBands = 72;

// Nominal bands of about 16 MiB per host plane: 16 .. 64 bands, and at least
// 8 rows each.
int host_band_count(int64_t L, size_t hrow)
{
    const int64_t by_bytes = (int64_t)(((size_t)L * hrow) >> 24);
    const int64_t k = std::min<int64_t>(std::max<int64_t>(by_bytes, 16), 64);
    return (int)std::min<int64_t>(k, L / 8);
}

// Band starts and sizes (rows): nominal bands, except that where the lattice
// is large enough the first and last three bands are 1/8, 1/4 and 1/2 of the
// nominal size (mirrored), so that the first half-sweep waits for little data
// and the last copies out are short.  Returns the number of bands (>= 3, no
// empty band, at most kMaxHostBands).
int host_bands(int64_t L, size_t hrow, int64_t *b0, int64_t *br)
{
    const int nk = host_band_count(L, hrow);
    const int64_t per = (L + nk - 1) / nk;
    const int64_t ramp[3] = {per / 8, per / 4, per / 2};
    int K = 0;
    int64_t at = 0;
    auto add = [&](int64_t rows) {
        b0[K] = at;
        br[K] = rows;
        at += rows;
        ++K;
    };
    if (per >= 64 && L >= 4 * per) {
        const int64_t ends = ramp[0] + ramp[1] + ramp[2];
        for (int i = 0; i < 3; ++i) add(ramp[i]);
        while (at < L - ends) add(std::min<int64_t>(per, L - ends - at));
        for (int i = 2; i >= 0; --i) add(ramp[i]);
    } else {
        while (at < L) add(std::min<int64_t>(per, L - at));
    }
    return K;
}

// The events of the banded host path, per device, made on first use; the
// caller holds g_dev.host_mu while it enqueues, so no two calls interleave their
// records of them (a wait refers to the record made before it is enqueued).
constexpr int kHostEvents = 3 * kMaxHostBands + 2;

int host_events(int dev, cudaEvent_t **ev)
{
    if (g_dev.host_ev[dev] == nullptr) {
        cudaEvent_t *e = new cudaEvent_t[kHostEvents];
        for (int i = 0; i < kHostEvents; ++i) {
            cudaError_t r = cudaEventCreateWithFlags(&e[i], cudaEventDisableTiming);
            if (r != cudaSuccess) {
                for (int j = 0; j < i; ++j) cudaEventDestroy(e[j]);
                delete[] e;
                return cuda_fail(r, "event create");
            }
        }
        g_dev.host_ev[dev] = e;
    }
    *ev = g_dev.host_ev[dev];
    return ISING_OK;
}

// Queues one banded host sweep: stream `s` starts and ends it (it may be a
// stream in capture), `cmp` and `out` are the compute and copy-out streams,
// `ev` the event pool (caller holds g_dev.host_mu).
int enqueue_banded(const ising_lattice_t *dev, char *host[2], char *stage, size_t hrow, const Accept &acc,
                   const RoundKeys &rk, uint64_t t, int64_t *trace_dev, int64_t *trace_host, cudaStream_t s,
                   cudaStream_t cmp, cudaStream_t out, cudaEvent_t *ev)
{
    const int64_t L = dev->L;
    int64_t b0[kMaxHostBands], br[kMaxHostBands];
    const int K = host_bands(L, hrow, b0, br);
    int rc = ISING_OK;
    cudaError_t e = cudaSuccess;
    cudaEvent_t start = ev[0], end = ev[1], *ev_in = ev + 2, *ev_flush = ev_in + K;  // 2K flush events
    const bool bits = stage != nullptr;
    char *devp[2] = {(char *)dev->black, (char *)dev->white};
    char *stg[2] = {stage, bits ? stage + (size_t)L * hrow : nullptr};
    const size_t pitch = (size_t)dev->row_stride_bytes;
    const int64_t stride_words = dev->row_stride_bytes / 8;
    auto copy = [&](int c, int k, bool in, cudaStream_t st) {
        char *d = devp[c] + b0[k] * pitch, *h = host[c] + b0[k] * hrow;
        if (bits) {
            char *g = stg[c] + b0[k] * hrow;
            return in ? cudaMemcpyAsync(g, h, (size_t)br[k] * hrow, cudaMemcpyHostToDevice, st)
                      : cudaMemcpyAsync(h, g, (size_t)br[k] * hrow, cudaMemcpyDeviceToHost, st);
        }
        return in ? cudaMemcpy2DAsync(d, pitch, h, hrow, hrow, (size_t)br[k], cudaMemcpyHostToDevice, st)
                  : cudaMemcpy2DAsync(h, hrow, d, pitch, hrow, (size_t)br[k], cudaMemcpyDeviceToHost, st);
    };
    // bits mode: staged band -> MSC4 band (after its copy in) and back (before its copy out)
    // bits mode: staged plane band -> MSC4 band (as a conversion job)
    auto unpack_job = [&](int c, int k) {
        return ConvJob{stg[c] + b0[k] * hrow, devp[c] + b0[k] * pitch, br[k]};
    };
    e = cudaEventRecord(start, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cmp, start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(out, start, 0);
    // copy-in order: white K-1, 0, 1, black 0, then white k+1 and black k
    // (k = 1 .. K-2), black K-1; ev_in[k] follows black band k, after which
    // every plane band that black k reads is in
    auto in_black = [&](int k) {
        cudaError_t r = copy(0, k, true, s);
        return r == cudaSuccess ? cudaEventRecord(ev_in[k], s) : r;
    };
    if (e == cudaSuccess) e = copy(1, K - 1, true, s);
    if (e == cudaSuccess) e = copy(1, 0, true, s);
    if (e == cudaSuccess) e = copy(1, 1, true, s);
    if (e == cudaSuccess) e = in_black(0);
    for (int k = 1; k + 1 < K && e == cudaSuccess; ++k) {
        if (k + 1 < K - 1) e = copy(1, k + 1, true, s);
        if (e == cudaSuccess) e = in_black(k);
    }
    if (e == cudaSuccess) e = in_black(K - 1);
    if (e == cudaSuccess && trace_dev) e = cudaMemsetAsync(trace_dev, 0, 2 * sizeof(int64_t), cmp);
    if (e != cudaSuccess) return cuda_fail(e, "host sweep: copy in");
    // compute.  Plane bands that are final wait in `pend` and are flushed to
    // the copy-out stream behind one event: in MSC4 mode after every
    // half-sweep; in bits mode after every white half-sweep, packed by one
    // conversion launch for all of them (black k and white k-1).  In bits mode
    // black k first unpacks, in one launch, its own band and the white bands
    // it is the first to need, in their copy-in order (K-1, 0, 1, .., K-2):
    // the first min(k + 3, K) of that order.  Fewer, larger launches: each
    // launch leaves the SMs partly idle at its start and end.
    int unpacked = 0, n_flush = 0, npend = 0;
    int pend_c[kMaxConvJobs], pend_k[kMaxConvJobs];
    auto flush = [&]() -> int {
        if (npend == 0) return ISING_OK;
        cudaError_t r = cudaSuccess;
        if (bits) {
            ConvJob jobs[kMaxConvJobs];
            for (int i = 0; i < npend; ++i) {
                const int c = pend_c[i], k = pend_k[i];
                jobs[i] = ConvJob{devp[c] + b0[k] * pitch, stg[c] + b0[k] * hrow, br[k]};
            }
            r = msc4_to_bits_multi(jobs, npend, stride_words, L, cmp);
        }
        cudaEvent_t f = ev_flush[n_flush++];
        if (r == cudaSuccess) r = cudaEventRecord(f, cmp);
        if (r == cudaSuccess) r = cudaStreamWaitEvent(out, f, 0);
        for (int i = 0; i < npend && r == cudaSuccess; ++i) r = copy(pend_c[i], pend_k[i], false, out);
        npend = 0;
        return r == cudaSuccess ? ISING_OK : cuda_fail(r, "host sweep: copy out");
    };
    auto black = [&](int k) -> int {
        cudaError_t r = cudaStreamWaitEvent(cmp, ev_in[k], 0);
        if (r == cudaSuccess && bits) {
            ConvJob jobs[kMaxConvJobs];
            int n = 0;
            for (; unpacked < std::min(k + 3, K); ++unpacked)
                jobs[n++] = unpack_job(1, unpacked == 0 ? K - 1 : unpacked - 1);
            jobs[n++] = unpack_job(0, k);
            r = bits_to_msc4_multi(jobs, n, stride_words, L, cmp);
        }
        if (r != cudaSuccess) return cuda_fail(r, "host sweep: unpack");
        int x = band_half_sweep_impl(dev, acc, rk, 0, t, b0[k], br[k], nullptr, cmp);
        if (x) return x;
        pend_c[npend] = 0;
        pend_k[npend++] = k;
        return bits ? ISING_OK : flush();
    };
    auto white = [&](int k) -> int {
        int x = band_half_sweep_impl(dev, acc, rk, 1, t, b0[k], br[k], trace_dev, cmp);
        if (x) return x;
        pend_c[npend] = 1;
        pend_k[npend++] = k;
        return flush();
    };
    rc = black(0);
    if (!rc) rc = black(1);
    for (int k = 2; k < K && !rc; ++k) {
        rc = black(k);
        if (!rc) rc = white(k - 1);
    }
    if (!rc) rc = white(K - 1);
    if (!rc) rc = white(0);
    if (rc) return rc;
    if (trace_host != nullptr)
        e = cudaMemcpyAsync(trace_host, trace_dev, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, out);
    if (e == cudaSuccess) e = cudaEventRecord(end, out);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, end, 0);
    return e == cudaSuccess ? ISING_OK : cuda_fail(e, "host sweep: copy out");
}

// One banded host sweep.  The schedule (about 4 launches and 4 copies per
// band, with cross-stream events) is captured on the library's capture stream
// and replayed as a CUDA graph on `s`: the executable graph of the previous
// call is updated in place (new sweep index, keys, buffers) where the
// topology is the same, else instantiated anew.  Capture and update run on the
// host while the GPU still executes the previous call.  Any failure of the
// capture path falls back to launching the schedule directly on `s`.
int sweep_host_banded(const ising_lattice_t *dev, char *host[2], char *stage, size_t hrow, const Accept &acc,
                      const RoundKeys &rk, uint64_t t, int64_t *trace_dev, int64_t *trace_host, cudaStream_t s)
{
    cudaStream_t cmp = nullptr, out = nullptr, cap = nullptr;
    int rc = aux_streams(&cmp, &out, &cap);
    if (rc) return rc;
    int devi = 0;
    cudaError_t e = cudaGetDevice(&devi);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(g_dev.host_mu);
    cudaEvent_t *ev = nullptr;
    rc = host_events(devi, &ev);
    if (rc) return rc;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const int crc = enqueue_banded(dev, host, stage, hrow, acc, rk, t, trace_dev, trace_host, cap, cmp, out, ev);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(cap, &g);
        if (crc == ISING_OK && ce == cudaSuccess && g != nullptr) {
            cudaGraphExec_t &x = g_dev.host_exec[devi];
            bool ready = false;
            if (x != nullptr) {
                cudaGraphExecUpdateResultInfo info;
                ready = cudaGraphExecUpdate(x, g, &info) == cudaSuccess;
                if (!ready) {
                    cudaGetLastError();
                    cudaGraphExecDestroy(x);
                    x = nullptr;
                }
            }
            if (!ready) {
                ready = cudaGraphInstantiate(&x, g, 0) == cudaSuccess;
                if (!ready) x = nullptr;
            }
            cudaGraphDestroy(g);
            if (ready) {
                e = cudaGraphLaunch(x, s);
                return e == cudaSuccess ? ISING_OK : cuda_fail(e, "host sweep: graph launch");
            }
        } else if (g != nullptr) {
            cudaGraphDestroy(g);
        }
        cudaGetLastError();  // the capture path failed: clear its error, launch directly
    }
    return enqueue_banded(dev, host, stage, hrow, acc, rk, t, trace_dev, trace_host, s, cmp, out, ev);
}

}  // namespace

ISING_API int ising_sweep_host(const ising_lattice_t *dev, void *black_host, void *white_host, double beta,
                               int64_t n_sweeps, uint64_t seed, uint64_t sweep_offset, int64_t *trace_dev,
                               int64_t *trace_host, ising_stream_t stream)
{
    int rc = check_lattice(dev);
    if (rc) return rc;
    if (black_host == nullptr || white_host == nullptr) return fail(ISING_EINVAL, "host planes are NULL");
    if (trace_host != nullptr && trace_dev == nullptr)
        return fail(ISING_EINVAL, "trace_host needs trace_dev as device staging");
    size_t row = 0;
    row_bytes_of(dev->L, dev->layout, &row);
    cudaStream_t s = (cudaStream_t)stream;
    if (n_sweeps == 1 && dev->layout == ISING_MSC4) {
        Accept acc;
        uint64_t T[5];
        rc = build_accept(beta, &acc, T);
        if (rc) return rc;
        if (trace_dev != nullptr) {
            rc = check_device_range(trace_dev, 2 * sizeof(int64_t), "trace");
            if (rc) return rc;
        }
        char *host[2] = {(char *)black_host, (char *)white_host};
        return sweep_host_banded(dev, host, nullptr, row, acc, make_round_keys(seed), sweep_offset, trace_dev,
                                 trace_host, s);
    }
    void *host[2] = {black_host, white_host};
    void *devp[2] = {dev->black, dev->white};
    for (int c = 0; c < 2; ++c) {
        cudaError_t e = cudaMemcpy2DAsync(devp[c], (size_t)dev->row_stride_bytes, host[c], row, row, (size_t)dev->L,
                                          cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    }
    rc = ising_sweep(dev, beta, n_sweeps, seed, sweep_offset, trace_dev, stream);
    if (rc) return rc;
    for (int c = 0; c < 2; ++c) {
        cudaError_t e = cudaMemcpy2DAsync(host[c], row, devp[c], (size_t)dev->row_stride_bytes, row, (size_t)dev->L,
                                          cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
    }
    if (trace_host != nullptr && n_sweeps > 0) {
        cudaError_t e = cudaMemcpyAsync(trace_host, trace_dev, (size_t)n_sweeps * 2 * sizeof(int64_t),
                                        cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "trace copy");
    }
    return ISING_OK;
}

namespace {

int check_msc4_bits(const ising_lattice_t *lat, const void *black_bits, const void *white_bits, size_t *plane_bits)
{
    int rc = check_lattice(lat);
    if (rc) return rc;
    if (lat->layout != ISING_MSC4) return fail(ISING_EINVAL, "the bit-packed format converts MSC4 lattices");
    rc = ising_bits_bytes(lat->L, plane_bits);
    if (rc) return rc;
    if (black_bits == nullptr || white_bits == nullptr) return fail(ISING_EINVAL, "bit planes are NULL");
    if (((uintptr_t)black_bits | (uintptr_t)white_bits) % 4 != 0)
        return fail(ISING_EINVAL, "bit planes must be 4-byte aligned");
    return ISING_OK;
}

}  // namespace

ISING_API int ising_bits_bytes(int64_t L, size_t *bytes_per_plane)
{
    if (bytes_per_plane == nullptr) return fail(ISING_EINVAL, "bytes_per_plane is NULL");
    size_t row = 0;
    int rc = row_bytes_of(L, ISING_MSC4, &row);  // L even, L % 64 == 0
    if (rc) return rc;
    *bytes_per_plane = (size_t)L * (size_t)(L / 16);
    return ISING_OK;
}

ISING_API int ising_msc4_to_bits(const ising_lattice_t *msc4, void *black_bits, void *white_bits,
                                 ising_stream_t stream)
{
    size_t nb = 0;
    int rc = check_msc4_bits(msc4, black_bits, white_bits, &nb);
    if (rc) return rc;
    rc = check_device_range(black_bits, nb, "black bits");
    if (!rc) rc = check_device_range(white_bits, nb, "white bits");
    if (rc) return rc;
    const int64_t sw = msc4->row_stride_bytes / 8;
    cudaError_t e = msc4_to_bits((const uint64_t *)msc4->black, sw, (uint32_t *)black_bits, msc4->L, msc4->L,
                                 (cudaStream_t)stream);
    if (e == cudaSuccess)
        e = msc4_to_bits((const uint64_t *)msc4->white, sw, (uint32_t *)white_bits, msc4->L, msc4->L,
                         (cudaStream_t)stream);
    return e == cudaSuccess ? ISING_OK : cuda_fail(e, "to-bits launch");
}

ISING_API int ising_bits_to_msc4(const void *black_bits, const void *white_bits, const ising_lattice_t *msc4,
                                 ising_stream_t stream)
{
    size_t nb = 0;
    int rc = check_msc4_bits(msc4, black_bits, white_bits, &nb);
    if (rc) return rc;
    rc = check_device_range(black_bits, nb, "black bits");
    if (!rc) rc = check_device_range(white_bits, nb, "white bits");
    if (rc) return rc;
    const int64_t sw = msc4->row_stride_bytes / 8;
    cudaError_t e = bits_to_msc4((const uint32_t *)black_bits, (uint64_t *)msc4->black, sw, msc4->L, msc4->L,
                                 (cudaStream_t)stream);
    if (e == cudaSuccess)
        e = bits_to_msc4((const uint32_t *)white_bits, (uint64_t *)msc4->white, sw, msc4->L, msc4->L,
                         (cudaStream_t)stream);
    return e == cudaSuccess ? ISING_OK : cuda_fail(e, "from-bits launch");
}

ISING_API int ising_sweep_host_bits(const ising_lattice_t *dev, void *black_host, void *white_host, void *stage_dev,
                                    double beta, int64_t n_sweeps, uint64_t seed, uint64_t sweep_offset,
                                    int64_t *trace_dev, int64_t *trace_host, ising_stream_t stream)
{
    size_t nb = 0;
    int rc = check_msc4_bits(dev, black_host, white_host, &nb);
    if (rc) return rc;
    if (stage_dev == nullptr || (uintptr_t)stage_dev % 16 != 0)
        return fail(ISING_EINVAL, "stage_dev must be a 16-byte aligned device buffer");
    rc = check_device_range(stage_dev, 2 * nb, "stage");
    if (rc) return rc;
    if (n_sweeps < 0) return fail(ISING_EINVAL, "n_sweeps = %lld < 0", (long long)n_sweeps);
    if (trace_host != nullptr && trace_dev == nullptr)
        return fail(ISING_EINVAL, "trace_host needs trace_dev as device staging");
    if (trace_dev != nullptr && n_sweeps > 0) {
        rc = check_device_range(trace_dev, (size_t)n_sweeps * 2 * sizeof(int64_t), "trace");
        if (rc) return rc;
    }
    Accept acc;
    uint64_t T[5];
    rc = build_accept(beta, &acc, T);
    if (rc) return rc;
    const size_t hrow = (size_t)(dev->L / 16);
    cudaStream_t s = (cudaStream_t)stream;
    char *host[2] = {(char *)black_host, (char *)white_host};
    char *stg[2] = {(char *)stage_dev, (char *)stage_dev + nb};
    if (n_sweeps == 1)
        return sweep_host_banded(dev, host, (char *)stage_dev, hrow, acc, make_round_keys(seed), sweep_offset,
                                 trace_dev, trace_host, s);
    for (int c = 0; c < 2; ++c) {
        cudaError_t e = cudaMemcpyAsync(stg[c], host[c], nb, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    }
    rc = ising_bits_to_msc4(stg[0], stg[1], dev, stream);
    if (!rc) rc = ising_sweep(dev, beta, n_sweeps, seed, sweep_offset, trace_dev, stream);
    if (!rc) rc = ising_msc4_to_bits(dev, stg[0], stg[1], stream);
    if (rc) return rc;
    for (int c = 0; c < 2; ++c) {
        cudaError_t e = cudaMemcpyAsync(host[c], stg[c], nb, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
    }
    if (trace_host != nullptr && n_sweeps > 0) {
        cudaError_t e = cudaMemcpyAsync(trace_host, trace_dev, (size_t)n_sweeps * 2 * sizeof(int64_t),
                                        cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "trace copy");
    }
    return ISING_OK;
}

ISING_API int ising_observables(const ising_lattice_t *lat, int64_t *out_dev, ising_stream_t stream)
{
    int rc = check_lattice(lat);
    if (rc) return rc;
    rc = check_device_range(out_dev, 2 * sizeof(int64_t), "out");
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(out_dev, 0, 2 * sizeof(int64_t), s);
    if (e != cudaSuccess) return cuda_fail(e, "observables memset");
    e = lat->layout == ISING_MSC4
            ? msc4_observables((const uint64_t *)lat->black, (const uint64_t *)lat->white, lat->L,
                               lat->row_stride_bytes / 8, (long long *)out_dev, s)
            : int8_observables((const int8_t *)lat->black, (const int8_t *)lat->white, lat->L, lat->row_stride_bytes,
                               (long long *)out_dev, s);
    return e == cudaSuccess ? ISING_OK : cuda_fail(e, "observables launch");
}

static int check_pair(const ising_lattice_t *a, int32_t la, const ising_lattice_t *b, int32_t lb)
{
    int rc = check_lattice(a);
    if (rc) return rc;
    rc = check_lattice(b);
    if (rc) return rc;
    if (a->layout != la || b->layout != lb) return fail(ISING_EINVAL, "wrong layouts for conversion");
    if (a->L != b->L) return fail(ISING_EINVAL, "lattice sizes differ");
    return ISING_OK;
}

ISING_API int ising_pack(const ising_lattice_t *int8_src, const ising_lattice_t *msc4_dst, ising_stream_t stream)
{
    int rc = check_pair(int8_src, ISING_INT8, msc4_dst, ISING_MSC4);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    for (int c = 0; c < 2; ++c) {
        cudaError_t e = msc4_pack((const int8_t *)(c ? int8_src->white : int8_src->black), int8_src->row_stride_bytes,
                                  (uint64_t *)(c ? msc4_dst->white : msc4_dst->black), msc4_dst->row_stride_bytes / 8,
                                  int8_src->L, s);
        if (e != cudaSuccess) return cuda_fail(e, "pack launch");
    }
    return ISING_OK;
}

ISING_API int ising_unpack(const ising_lattice_t *msc4_src, const ising_lattice_t *int8_dst, ising_stream_t stream)
{
    int rc = check_pair(msc4_src, ISING_MSC4, int8_dst, ISING_INT8);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    for (int c = 0; c < 2; ++c) {
        cudaError_t e = msc4_unpack((const uint64_t *)(c ? msc4_src->white : msc4_src->black),
                                    msc4_src->row_stride_bytes / 8, (int8_t *)(c ? int8_dst->white : int8_dst->black),
                                    int8_dst->row_stride_bytes, msc4_src->L, s);
        if (e != cudaSuccess) return cuda_fail(e, "unpack launch");
    }
    return ISING_OK;
}

ISING_API int ising_rng_probe(uint64_t n_blocks, uint64_t seed, uint64_t t, int32_t colour, uint32_t T3,
                              uint64_t *count_dev, ising_stream_t stream)
{
    if (colour != 0 && colour != 1) return fail(ISING_EINVAL, "colour must be 0 or 1");
    if (n_blocks > (uint64_t(1) << 34)) return fail(ISING_EINVAL, "n_blocks must be at most 2^34");
    int rc = check_device_range(count_dev, sizeof(uint64_t), "count");
    if (rc) return rc;
    if (n_blocks == 0) return ISING_OK;
    cudaError_t e = rng_probe(n_blocks, make_round_keys(seed), (uint32_t)t,
                              counter_word3(colour, kPurposeMetropolis, t), T3, (unsigned long long *)count_dev,
                              (cudaStream_t)stream);
    return e == cudaSuccess ? ISING_OK : cuda_fail(e, "rng probe launch");
}

ISING_API int ising_mulwide_probe(int32_t form, uint32_t iters, uint64_t *sink_dev, uint64_t *multiplies,
                                  ising_stream_t stream)
{
    if (form != 0 && form != 1) return fail(ISING_EINVAL, "form must be 0 or 1");
    if (iters == 0 || multiplies == nullptr) return fail(ISING_EINVAL, "iters must be > 0 and multiplies non-NULL");
    int rc = check_device_range(sink_dev, sizeof(uint64_t), "sink");
    if (rc) return rc;
    cudaError_t e = mulwide_probe(form, iters, (unsigned long long *)sink_dev, multiplies, (cudaStream_t)stream);
    return e == cudaSuccess ? ISING_OK : cuda_fail(e, "multiply probe launch");
}

}  // extern "C"
