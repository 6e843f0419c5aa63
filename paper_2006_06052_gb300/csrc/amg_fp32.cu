// Instantiation of the device AMG and Schur preconditioners for the
// fp32 storage form (one translation unit per form so they build in
// parallel).
#include "amg_dev.cuh"

namespace gbs {

std::unique_ptr<DevPrecond> make_amg_fp32(const HAmg& H, const PrecondOptions& o, cudaStream_t s) {
  auto p = std::make_unique<AmgPrecond<1>>();
  p->init(H, o, s);
  return p;
}

std::unique_ptr<DevPrecond> make_schur_fp32(const HSchur& Sc, const HAmg& HA, const HAmg& HS,
                                           const PrecondOptions& o, cudaStream_t s) {
  auto p = std::make_unique<SchurPrecond<1>>();
  p->init(Sc, HA, HS, o, s);
  return p;
}

}  // namespace gbs
