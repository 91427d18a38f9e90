// Tensor-core NIF of width 128 (the workloads' network) and the dispatch over
// widths; the kernel itself is in nif_tc.cuh, widths 64 and 32 are compiled
// in nif_tc_small.cu.
#include "nif_tc.cuh"

namespace ptk {
namespace tcnif {

static_assert(Layout<128, 3>::slots == 3 && Layout<128, 5>::slots == 1 && Layout<128, 6>::slots < 1,
              "residency of the width-128 network: three slots up to L = 3, none from L = 6");
static_assert(max_layers<128>() == 5 && max_layers<64>() == 8 && max_layers<32>() == 8, "supported depths");

PT_NIF_TC_WIDTH(128)

}  // namespace tcnif

bool nif_tc_supported(int F, int H, int L)
{
    using namespace tcnif;
    if (F != kF || L < 1) return false;
    switch (H) {
    case 128: return L <= max_layers<128>();
    case 64: return L <= max_layers<64>();
    case 32: return L <= max_layers<32>();
    default: return false;
    }
}

bool pack_nif_tc_image(const float* params, int F, int H, int L, std::vector<unsigned char>& out)
{
    using namespace tcnif;
    if (!nif_tc_supported(F, H, L)) return false;
    switch (H) {
    case 128: return NifTcWidth<128>::pack(params, L, out);
    case 64: return NifTcWidth<64>::pack(params, L, out);
    default: return NifTcWidth<32>::pack(params, L, out);
    }
}

cudaError_t launch_nif_tc(const unsigned char* image, int H, int L, const NifEvalParams& np, int mode, int sm_count,
                          cudaStream_t s)
{
    using namespace tcnif;
    TcParams p = {};
    p.image = image;
    p.uv = np.uv;
    p.rgb = np.rgb;
    p.n = np.n;
    p.esc = np.esc;
    p.esc_count = np.esc_count;
    p.esc_cap = np.esc_cap;
    p.slot_L = np.slot_L;
    p.accumulate = np.accumulate;
    p.err = np.err;
    p.stats = np.stats;
    switch (H) {
    case 128: return NifTcWidth<128>::launch(L, p, mode, sm_count, s);
    case 64: return NifTcWidth<64>::launch(L, p, mode, sm_count, s);
    case 32: return NifTcWidth<32>::launch(L, p, mode, sm_count, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t repack_nif_tc_image(const float* params, int H, int L, unsigned char* image, cudaStream_t s)
{
    using namespace tcnif;
    switch (H) {
    case 128: return NifTcWidth<128>::repack(params, L, image, s);
    case 64: return NifTcWidth<64>::repack(params, L, image, s);
    case 32: return NifTcWidth<32>::repack(params, L, image, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ptk
