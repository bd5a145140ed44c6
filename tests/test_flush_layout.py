"""The consumer kernel's flush order (tree_layout.h flush_node): every inner node of a
depth-D tree at exactly one position, and each group's positions holding exactly that
group's nodes -- the three nodes of each of its GS bottom subtrees, then the inner nodes
of the subtree above those roots -- with the nodes above all groups last.  The kernel
keeps the group's accumulators in registers and flushes them with the group, so a node
in the wrong group would be added into phi before all of its slot sums were complete."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2511_09376_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "tree_layout.h"
int main() {
    for (int D = 2; D <= 8; ++D) {
        std::printf("%d %d %d %d", D, wdf::gather_group(D), wdf::flush_group_len(D), wdf::flush_len(D));
        for (int i = 0; i < wdf::flush_len(D); ++i) std::printf(" %d", wdf::flush_node(D, i));
        std::printf("\n");
    }
    return 0;
}
"""


def _ancestors(v):
    out = []
    while v > 0:
        v = (v - 1) // 2
        out.append(v)
    return out


def test_flush_order_groups_and_covers_every_node(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "flush.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "flush"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, lines):
        D, GS, GL, FL, *pos = map(int, line.split())
        NS, NI = 1 << (D - 2), (1 << D) - 1
        NG = NS // GS
        assert FL % 8 == 0 and GL % 8 == 0 and len(pos) == FL
        assert sorted(v for v in pos if v >= 0) == list(range(NI)), D  # each node once
        roots = [NS - 1 + s for s in range(NS)]
        for g in range(NG):
            block = [v for v in pos[g * GL:(g + 1) * GL] if v >= 0]
            mine = roots[g * GS:(g + 1) * GS]
            bottom = [n for r in mine for n in (r, 2 * r + 1, 2 * r + 2)]
            assert block[:3 * GS] == bottom, (D, g)  # subtree by subtree, root first
            # the nodes above this group's roots that no other group's root has
            upper = set()
            for r in mine:
                upper.update(_ancestors(r))
            for r in roots[:g * GS] + roots[(g + 1) * GS:]:
                upper.difference_update(_ancestors(r))
            assert block[3 * GS:] == sorted(upper), (D, g)  # heap order
        top = [v for v in pos[NG * GL:] if v >= 0]
        assert top == list(range(NG - 1)), D
        if NG == 1:  # one group: all bottom nodes, then all nodes above them
            assert [v for v in pos if v >= 0][3 * NS:] == list(range(NS - 1))
