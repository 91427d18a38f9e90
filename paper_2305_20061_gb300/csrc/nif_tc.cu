// Tensor-core NIF of width 128 (the workloads' network) and the dispatch over
// network shapes; the kernel itself is in nif_tc.cuh, widths 64 and 32 are
// compiled in nif_tc_small.cu, width 256 and the paper's skip network in
// nif_tc_shapes.cu.
#include "nif_tc.cuh"

namespace ptk {
namespace tcnif {

static_assert(Layout<64, 128, 3, 0>::slots == 3 && Layout<64, 128, 5, 0>::slots == 1 &&
                  Layout<64, 128, 6, 0>::slots < 1,
              "residency of the width-128 network: three slots up to L = 3, none from L = 6");
static_assert(max_layers<128>() == 5 && max_layers<64>() == 8 && max_layers<32>() == 8 && max_layers<256>() == 1,
              "supported depths");
static_assert(Layout<kPaperF, kPaperH, kPaperL, kPaperS>::slots == 3, "the paper's network keeps three slots");

PT_NIF_TC_WIDTH(128)

}  // namespace tcnif

bool nif_tc_supported(int F, int H, int L, int S)
{
    using namespace tcnif;
    if (F == kPaperF && H == kPaperH && L == kPaperL && S == kPaperS) return true;
    if (F != 64 || S != 0 || L < 1) return false;
    switch (H) {
    case 256: return L <= max_layers<256>();
    case 128: return L <= max_layers<128>();
    case 64: return L <= max_layers<64>();
    case 32: return L <= max_layers<32>();
    default: return false;
    }
}

bool pack_nif_tc_image(const float* params, int F, int H, int L, int S, std::vector<unsigned char>& out)
{
    using namespace tcnif;
    if (!nif_tc_supported(F, H, L, S)) return false;
    if (S) return pack_paper_skip(params, out);
    switch (H) {
    case 256: return NifTcWidth<256>::pack(params, L, out);
    case 128: return NifTcWidth<128>::pack(params, L, out);
    case 64: return NifTcWidth<64>::pack(params, L, out);
    default: return NifTcWidth<32>::pack(params, L, out);
    }
}

cudaError_t launch_nif_tc(const unsigned char* image, int F, int H, int L, int S, const NifEvalParams& np, int mode,
                          int sm_count, cudaStream_t s)
{
    using namespace tcnif;
    if (!nif_tc_supported(F, H, L, S)) return cudaErrorInvalidValue;
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
    if (S) return launch_paper_skip(p, mode, sm_count, s);
    switch (H) {
    case 256: return NifTcWidth<256>::launch(L, p, mode, sm_count, s);
    case 128: return NifTcWidth<128>::launch(L, p, mode, sm_count, s);
    case 64: return NifTcWidth<64>::launch(L, p, mode, sm_count, s);
    default: return NifTcWidth<32>::launch(L, p, mode, sm_count, s);
    }
}

cudaError_t repack_nif_tc_image(const float* params, int F, int H, int L, int S, unsigned char* image, cudaStream_t s)
{
    using namespace tcnif;
    if (!nif_tc_supported(F, H, L, S)) return cudaErrorInvalidValue;
    if (S) return repack_paper_skip(params, image, s);
    switch (H) {
    case 256: return NifTcWidth<256>::repack(params, L, image, s);
    case 128: return NifTcWidth<128>::repack(params, L, image, s);
    case 64: return NifTcWidth<64>::repack(params, L, image, s);
    default: return NifTcWidth<32>::repack(params, L, image, s);
    }
}

}  // namespace ptk
