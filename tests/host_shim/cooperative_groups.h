// Host stand-in for the cluster part of cooperative_groups used by the four-CTA FFT
// (fft_cluster.cuh): the caller emulates the CTAs of one cluster one after another, sets
// host_cluster_rank to the CTA being run and host_cta_base[q] to CTA q's shared-memory buffer
// (test use only).
#pragma once

inline int host_cluster_rank = 0;
inline char* host_cta_base[8] = {};

namespace cooperative_groups {
struct HostCluster {
  unsigned block_rank() const { return (unsigned)host_cluster_rank; }
  void sync() const {}
  template <class T>
  T* map_shared_rank(T* p, int q) const {
    return reinterpret_cast<T*>(reinterpret_cast<char*>(p) - host_cta_base[host_cluster_rank] + host_cta_base[q]);
  }
};
inline HostCluster this_cluster() { return {}; }
}  // namespace cooperative_groups
