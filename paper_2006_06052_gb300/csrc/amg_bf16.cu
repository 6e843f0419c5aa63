// Instantiation of the device AMG and Schur preconditioners for the
// bf16 storage form (one translation unit per form so they build in
// parallel).
#include "amg_dev.cuh"

namespace gbs {

std::unique_ptr<DevPrecond> make_amg_bf16(const HAmg& H, const PrecondOptions& o, cudaStream_t s) {
  auto p = std::make_unique<AmgPrecond<2>>();
  p->init(H, o, s);
  return p;
}

std::unique_ptr<DevPrecond> make_schur_bf16(const HSchur& Sc, const HAmg& HA, const HAmg& HS,
                                           const PrecondOptions& o, cudaStream_t s) {
  auto p = std::make_unique<SchurPrecond<2>>();
  p->init(Sc, HA, HS, o, s);
  return p;
}

}  // namespace gbs
