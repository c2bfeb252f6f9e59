// fdd_noalloc.cu -- phase-rotate-and-sum for callers that cannot allocate.
//
// Some callers own every byte of device memory themselves: a host application
// whose framework pre-reserves the GPU in its own pool, or a real-time
// pipeline that forbids allocation once it has started.  They cannot create a
// plan (fdd_plan allocates its workspace).  fdd_dedisperse_spectra_static
// runs the same phase-rotate-and-sum kernel as fdd_dedisperse_spectra, but
// takes the parameters directly and keeps the per-channel phase table the
// kernel reads in the file-scope device array below instead of plan memory.
// Nothing is allocated on the device or the host: the table is written by a
// small kernel whose launch parameters carry the constants by value.
#include <atomic>

#include "fdd.h"
#include "fdd_internal.h"

namespace {

constexpr int kMaxChan = FDD_STATIC_MAX_CHAN;
constexpr int kMaxDevices = 64;
// Channels per table-fill launch: 240 constants of 16 bytes keep the launch
// parameters within the classic 4 KiB limit.
constexpr int kFillBlock = 240;

// The phase table (16 bytes per channel, 128 KiB).  Every GPU that loads the
// library holds it until the process exits, and every call shares it.
static __device__ __align__(256) fdd::PhaseConst g_phase_table[kMaxChan];

// Device address of g_phase_table, looked up once per device.  In host code
// the name g_phase_table is only a host-side stand-in, never a device address.
std::atomic<fdd::PhaseConst*> g_table_addr[kMaxDevices];

struct TableBlock {
  int first;
  int count;
  fdd::PhaseConst pc[kFillBlock];
};

__global__ void fill_table_kernel(fdd::PhaseConst* table, const TableBlock blk) {
  for (int i = threadIdx.x; i < blk.count; i += blockDim.x) table[blk.first + i] = blk.pc[i];
}

fdd_status table_address(int device, fdd::PhaseConst** out) {
  if (device < 0 || device >= kMaxDevices)
    return fdd::report_error(FDD_ERR_UNSUPPORTED, "device index beyond the supported range");
  fdd::PhaseConst* p = g_table_addr[device].load(std::memory_order_acquire);
  if (!p) {
    void* addr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&addr, g_phase_table);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fdd::report_error(FDD_ERR_CUDA, cudaGetErrorString(e));
    }
    p = static_cast<fdd::PhaseConst*>(addr);
    g_table_addr[device].store(p, std::memory_order_release);
  }
  *out = p;
  return FDD_OK;
}

}  // namespace

extern "C" fdd_status fdd_dedisperse_spectra_static(const fdd_params* p, const void* d_X,
                                                    int64_t x_pitch, int32_t n_series,
                                                    int32_t dm_first, int32_t n_dm, void* d_Y,
                                                    int64_t y_pitch, int32_t out_kind,
                                                    fdd_stream_t stream) {
  using fdd::report_error;
  if (!p) return report_error(FDD_ERR_INVALID_ARG, "params is NULL");
  if (!d_X || !d_Y) return report_error(FDD_ERR_INVALID_ARG, "NULL spectra pointer");
  if (p->n_chan > kMaxChan)
    return report_error(FDD_ERR_INVALID_ARG,
                        "n_chan exceeds FDD_STATIC_MAX_CHAN (8192) of the static phase table");
  if (p->mac_variant < 0 || p->mac_variant > FDD_MAC_VARIANTS)
    return report_error(FDD_ERR_INVALID_ARG, "mac_variant out of range");
  if (p->precision != FDD_PREC_FP32)
    return report_error(FDD_ERR_UNSUPPORTED,
                        "the allocation-free entry point runs the FP32 form only");
  // Channels, frequencies, DM list, transform length and chunking, checked
  // exactly as fdd_plan checks them.
  fdd::CoreGeometry g;
  fdd_status st = fdd::core_geometry(p, &g);
  if (st != FDD_OK) return st;
  if (!g.uniform)
    return report_error(FDD_ERR_UNSUPPORTED, "non-uniform DM lists are not supported");
  if (n_series < 1 || n_series > 65535)
    return report_error(FDD_ERR_INVALID_ARG, "n_series must be in [1, 65535]");
  if (dm_first < 0 || n_dm < 1 || dm_first + static_cast<int64_t>(n_dm) > p->n_dm)
    return report_error(FDD_ERR_INVALID_ARG, "trial range outside the DM list");
  if (out_kind != FDD_OUT_SPECTRA && out_kind != FDD_OUT_POWER)
    return report_error(FDD_ERR_INVALID_ARG, "out_kind must be FDD_OUT_SPECTRA or FDD_OUT_POWER");
  if (x_pitch < g.n_bins || y_pitch < g.n_bins)
    return report_error(FDD_ERR_INVALID_ARG, "pitches must be >= n_bins");

  const int variant = p->mac_variant ? p->mac_variant - 1 : fdd::mac_variant_for(p->n_dm, p->n_chan);
  if (fdd::mac_smem_bytes(variant, p->n_chan) > 227 * 1024)
    return report_error(FDD_ERR_UNSUPPORTED, "n_chan needs more shared memory than a CTA has");

  int device = -1;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return report_error(FDD_ERR_CUDA, cudaGetErrorString(e));
  fdd::PhaseConst* table = nullptr;
  if ((st = table_address(device, &table)) != FDD_OK) return st;
  e = fdd::mac_prepare(variant, p->n_chan);
  if (e != cudaSuccess) return report_error(FDD_ERR_CUDA, cudaGetErrorString(e));

  // Fill the table in stream order, kFillBlock channels per launch, with the
  // constants fdd_plan computes (the same function).
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  TableBlock blk;
  for (int c0 = 0; c0 < p->n_chan; c0 += kFillBlock) {
    blk.first = c0;
    blk.count = (p->n_chan - c0) < kFillBlock ? (p->n_chan - c0) : kFillBlock;
    for (int i = 0; i < blk.count; ++i)
      blk.pc[i] = fdd::phase_const(fdd::delay_rate(*p, g, c0 + i), static_cast<double>(g.L),
                                   g.dm0, g.ddm);
    fill_table_kernel<<<1, 256, 0, s>>>(table, blk);
    fdd::note_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return report_error(FDD_ERR_CUDA, cudaGetErrorString(e));
  }

  fdd::MacArgs m{};
  m.X = static_cast<const float2*>(d_X);
  m.x_chan_stride = x_pitch;
  m.x_series_stride = x_pitch * p->n_chan;
  m.pc = table;
  m.n_chan = p->n_chan;
  m.n_bins = static_cast<int>(g.n_bins);
  m.n_series = n_series;
  m.j_begin = dm_first;
  m.n_dm = n_dm;
  m.Y = d_Y;
  m.y_dm_stride = y_pitch;
  m.y_series_stride = y_pitch * n_dm;
  m.out_kind = out_kind == FDD_OUT_SPECTRA ? 1 : 2;
  m.scale = 1.0f;
  m.real_bin_a = -1;
  m.real_bin_b = -1;
  m.status = nullptr;  // no status word: see the header on timeouts
  e = fdd::launch_mac_fp32(m, variant, s);
  if (e != cudaSuccess) return report_error(FDD_ERR_CUDA, cudaGetErrorString(e));
  return FDD_OK;
}
