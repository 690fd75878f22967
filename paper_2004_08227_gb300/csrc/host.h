// host.h -- host-side declarations shared by the C-ABI translation units.
#pragma once
#include <string>
#include <vector>

namespace mplpp {

// Empty string on success, else a message.
std::string check_graph(int n, const std::vector<int> &eu, const std::vector<int> &ev);
std::string build_schedule(int kind, int n, const std::vector<int> &eu, const std::vector<int> &ev,
                           std::vector<int> &off, std::vector<int> &order);
std::string check_schedule(int n, const std::vector<int> &eu, const std::vector<int> &ev, const std::vector<int> &off,
                           const std::vector<int> &order);

}  // namespace mplpp
