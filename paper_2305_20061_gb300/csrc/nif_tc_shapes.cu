// Tensor-core NIF shapes beyond the workloads' family: one hidden layer of
// width 256 (the wide end of the model-size study, Section 4.6; deeper
// 256-wide networks do not stay resident) and the paper's own network
// (Section 3.2: 20 frequencies, four layers of 128, the second narrowed to
// 88 outputs and joined with the 40 features).  The kernel is in nif_tc.cuh.
#include "nif_tc.cuh"

namespace ptk {
namespace tcnif {

static_assert(Layout<64, 256, 1, 0>::slots == 2, "width 256: two slots of 64 KB and 256 TMEM columns");

PT_NIF_TC_WIDTH(256)

bool pack_paper_skip(const float* params, std::vector<unsigned char>& out)
{
    pack_image<kPaperF, kPaperH, kPaperL, kPaperS>(params, out);
    return true;
}

cudaError_t launch_paper_skip(const TcParams& p, int mode, int sm_count, cudaStream_t s)
{
    return launch_shape<kPaperF, kPaperH, kPaperL, kPaperS>(p, mode, sm_count, s);
}

cudaError_t repack_paper_skip(const float* params, unsigned char* image, cudaStream_t s)
{
    return repack_shape<kPaperF, kPaperH, kPaperL, kPaperS>(params, image, s);
}

}  // namespace tcnif
}  // namespace ptk
