// fdd_noalloc.cu -- phase-rotate-and-sum for callers that cannot allocate.
//
// Some callers own every byte of device memory themselves: a host application
// whose framework pre-reserves the GPU in its own pool, or a real-time
// pipeline that forbids allocation once it has started.  They cannot create a
// plan (fdd_plan allocates its workspace).  fdd_dedisperse_spectra_static
// runs the same phase-rotate-and-sum kernel as fdd_dedisperse_spectra, but
// takes the parameters directly and keeps the per-channel phase table the
// kernel reads in the file-scope device array below instead of plan memory.
// Nothing is allocated on the device or the host: the table is filled from a
// small stack buffer with stream-ordered copies.
#include <atomic>
#include <cmath>
#include <limits>

#include "fdd.h"
#include "fdd_internal.h"

namespace {

constexpr int kMaxChan = FDD_STATIC_MAX_CHAN;
constexpr int kMaxDevices = 64;
constexpr int kCopyBlock = 256;  // channels per host-to-device copy of the table

// The phase table (16 bytes per channel, 128 KiB).  Every GPU that loads the
// library holds it until the process exits, and every call shares it.
static __device__ __align__(256) fdd::PhaseConst g_phase_table[kMaxChan];

// Device address of g_phase_table, looked up once per device.  In host code
// the name g_phase_table is only a host-side stand-in, never a device address.
std::atomic<fdd::PhaseConst*> g_table_addr[kMaxDevices];

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
  if (p->n_chan < 1) return report_error(FDD_ERR_INVALID_ARG, "n_chan must be >= 1");
  if (p->n_chan > kMaxChan)
    return report_error(FDD_ERR_INVALID_ARG,
                        "n_chan exceeds FDD_STATIC_MAX_CHAN (8192) of the static phase table");
  if (!(p->t_samp_s > 0.0) || !std::isfinite(p->t_samp_s))
    return report_error(FDD_ERR_INVALID_ARG, "t_samp_s must be > 0");
  if (!(p->dnu_mhz != 0.0) || !std::isfinite(p->dnu_mhz))
    return report_error(FDD_ERR_INVALID_ARG, "dnu_mhz must be nonzero");
  if (!(p->k_dm >= 0.0) || !std::isfinite(p->k_dm))
    return report_error(FDD_ERR_INVALID_ARG, "k_dm must be >= 0");
  if (!p->dm_list || p->n_dm < 1) return report_error(FDD_ERR_INVALID_ARG, "empty DM list");
  if (p->n_t < 2) return report_error(FDD_ERR_INVALID_ARG, "n_t must be >= 2");
  if (p->chunk_len < 0 || (p->chunk_len % 2) != 0)
    return report_error(FDD_ERR_INVALID_ARG, "chunk_len must be 0 or a positive even length");
  if (p->mac_variant < 0 || p->mac_variant > FDD_MAC_VARIANTS)
    return report_error(FDD_ERR_INVALID_ARG, "mac_variant out of range");
  if (p->precision != FDD_PREC_FP32)
    return report_error(FDD_ERR_UNSUPPORTED,
                        "the allocation-free entry point runs the FP32 form only");
  if (n_series < 1 || n_series > 65535)
    return report_error(FDD_ERR_INVALID_ARG, "n_series must be in [1, 65535]");
  if (dm_first < 0 || n_dm < 1 || dm_first + static_cast<int64_t>(n_dm) > p->n_dm)
    return report_error(FDD_ERR_INVALID_ARG, "trial range outside the DM list");
  if (out_kind != FDD_OUT_SPECTRA && out_kind != FDD_OUT_POWER)
    return report_error(FDD_ERR_INVALID_ARG, "out_kind must be FDD_OUT_SPECTRA or FDD_OUT_POWER");

  // Transform length as fdd_plan_geometry defines it.
  int64_t L = p->chunk_len;
  if (L == 0) {
    L = 2;
    while (L < p->n_t) L <<= 1;
  }
  const int64_t n_bins = L / 2 + 1;
  if (x_pitch < n_bins || y_pitch < n_bins)
    return report_error(FDD_ERR_INVALID_ARG, "pitches must be >= n_bins");
  if (static_cast<double>(n_bins - 1) * static_cast<double>(p->n_dm - 1) >= 4294967296.0)
    return report_error(FDD_ERR_UNSUPPORTED, "(n_bins-1)*(n_dm-1) must be below 2^32");

  // Channel frequencies, reference frequency and the uniform DM grid.
  double nu_max = -1.0;
  for (int c = 0; c < p->n_chan; ++c) {
    const double nu = p->nu_lo_mhz + p->dnu_mhz * c;
    if (!(nu > 0.0) || !std::isfinite(nu))
      return report_error(FDD_ERR_INVALID_ARG, "channel centre is not positive");
    nu_max = nu > nu_max ? nu : nu_max;
  }
  const double nu_ref = p->nu_ref_mhz == 0.0 ? nu_max : p->nu_ref_mhz;
  if (!(nu_ref >= nu_max) || !std::isfinite(nu_ref))
    return report_error(FDD_ERR_INVALID_ARG, "nu_ref_mhz is below the highest channel centre");
  const double kdm = p->k_dm == 0.0 ? 1.0 / 2.41e-4 : p->k_dm;
  double dm_max = 0.0;
  for (int j = 0; j < p->n_dm; ++j) {
    const double dm = p->dm_list[j];
    if (!(dm >= 0.0) || !std::isfinite(dm))
      return report_error(FDD_ERR_INVALID_ARG, "DMs must be finite and >= 0");
    dm_max = dm > dm_max ? dm : dm_max;
  }
  const double dm0 = p->dm_list[0];
  const double ddm = p->n_dm > 1 ? (p->dm_list[p->n_dm - 1] - dm0) / (p->n_dm - 1) : 0.0;
  const double tol = 4.0 * std::ldexp(std::numeric_limits<double>::epsilon(),
                                      std::ilogb(dm_max > 1.0 ? dm_max : 1.0));
  for (int j = 0; j < p->n_dm; ++j)
    if (std::fabs(p->dm_list[j] - (dm0 + j * ddm)) > tol)
      return report_error(FDD_ERR_UNSUPPORTED, "non-uniform DM lists are not supported");

  const int variant = p->mac_variant ? p->mac_variant - 1 : fdd::mac_variant_for(p->n_dm);
  if (fdd::mac_smem_bytes(variant, p->n_chan) > 227 * 1024)
    return report_error(FDD_ERR_UNSUPPORTED, "n_chan needs more shared memory than a CTA has");

  int device = -1;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return report_error(FDD_ERR_CUDA, cudaGetErrorString(e));
  fdd::PhaseConst* table = nullptr;
  fdd_status st = table_address(device, &table);
  if (st != FDD_OK) return st;
  e = fdd::mac_prepare(variant, p->n_chan);
  if (e != cudaSuccess) return report_error(FDD_ERR_CUDA, cudaGetErrorString(e));

  // Fill the table (stream-ordered; the stack buffer is consumed before each
  // pageable copy returns).
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  fdd::PhaseConst buf[kCopyBlock];
  for (int c0 = 0; c0 < p->n_chan; c0 += kCopyBlock) {
    const int nc = (p->n_chan - c0) < kCopyBlock ? (p->n_chan - c0) : kCopyBlock;
    for (int i = 0; i < nc; ++i) {
      const double nu = p->nu_lo_mhz + p->dnu_mhz * (c0 + i);
      const double rate = kdm * (1.0 / (nu * nu) - 1.0 / (nu_ref * nu_ref)) / p->t_samp_s;
      const uint64_t u = fdd::fixed64_phase_rate(dm0, rate, static_cast<double>(L));
      const uint64_t v = fdd::fixed64_phase_rate(ddm, rate, static_cast<double>(L));
      buf[i] = fdd::PhaseConst{static_cast<uint32_t>(u), static_cast<uint32_t>(u >> 32),
                               static_cast<uint32_t>(v), static_cast<uint32_t>(v >> 32)};
    }
    e = cudaMemcpyAsync(table + c0, buf, sizeof(fdd::PhaseConst) * nc, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return report_error(FDD_ERR_CUDA, cudaGetErrorString(e));
  }

  fdd::MacArgs m{};
  m.X = static_cast<const float2*>(d_X);
  m.x_chan_stride = x_pitch;
  m.x_series_stride = x_pitch * p->n_chan;
  m.pc = table;
  m.n_chan = p->n_chan;
  m.n_bins = static_cast<int>(n_bins);
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
  m.status = nullptr;
  e = fdd::launch_mac_fp32(m, variant, s);
  if (e != cudaSuccess) return report_error(FDD_ERR_CUDA, cudaGetErrorString(e));
  return FDD_OK;
}
