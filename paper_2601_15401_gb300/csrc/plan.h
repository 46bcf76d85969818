// Partition-tree plans of the k-input multiplier (Section V-C).
#pragma once
#include <string>
#include <vector>

namespace ckks {

struct PlanNode {
    int size = 0;                 // inputs below this node
    std::vector<int> children;    // >= 0: node index; < 0: leaf -1 - input index
    int mu = 0;                   // m - 1 rescales
    bool root = false;
};

struct Plan {
    int k = 0;
    std::string text;
    std::vector<PlanNode> nodes;  // post-order, root last
    int depth = 0;
    int rs_units = 0;
};

const char *table_ii_partition(int k);
// 0 ok, -1 parse error, -2 depth rule broken
int plan_build(Plan &P, int k, const char *partition);
void plan_levels(const Plan &P, int level, std::vector<int> &lvl_in, std::vector<int> &lvl_out,
                 std::vector<int> &polys);

}  // namespace ckks
