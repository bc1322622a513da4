"""The library's Coulomb term decoding (csrc/terms.cuh, index arithmetic
compiled here as plain C++) against the oracle's term lists, index by index:
bit-exact for the unmerged 4N^2 list and the spin-merged 3N^2 list, with the
reuse block of every term."""
import os
import shutil
import subprocess

import pytest

from oracle import thc as TH

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TERMS = os.path.join(ROOT, "paper_2409_12708_gb300", "csrc", "terms.cuh")

PROGRAM = r"""
#include <cstdio>
#include "@TERMS@"
int main() {
    const int Ns[] = {1, 2, 3, 5};
    for (int N : Ns)
        for (int merge = 0; merge < 2; ++merge) {
            std::printf("count %d %d %ld\n", N, merge, thc::coulomb_terms(N, merge));
            for (long t = 0; t < thc::coulomb_terms(N, merge); ++t) {
                const thc::TermIdx d = thc::decode_coulomb(t, N, merge);
                std::printf("term %d %d %ld %d %d %d %d %.1f %ld\n", N, merge, t, d.mu, d.s, d.nu, d.sp, d.factor,
                            thc::coulomb_block(t, N, merge));
            }
        }
    return 0;
}
"""


@pytest.fixture(scope="module")
def decoded(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("terms")
    src, exe = d / "terms.cpp", d / "terms"
    src.write_text(PROGRAM.replace("@TERMS@", TERMS))
    subprocess.check_call([cxx, "-std=c++17", "-O1", str(src), "-o", str(exe)])
    counts, terms = {}, {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        f = line.split()
        if f[0] == "count":
            counts[(int(f[1]), int(f[2]))] = int(f[3])
        else:
            N, merge, t = int(f[1]), int(f[2]), int(f[3])
            terms[(N, merge, t)] = (int(f[4]), int(f[5]), int(f[6]), int(f[7]), float(f[8]), int(f[9]))
    return counts, terms


def test_term_counts(decoded):
    counts, _ = decoded
    for (N, merge), c in counts.items():
        assert c == TH.n_coulomb(N, bool(merge))


def test_unmerged_list_matches_the_oracle(decoded):
    _, terms = decoded
    L = 3
    for (N, merge, t), (mu, s, nu, sp, f, blk) in terms.items():
        if merge:
            continue
        assert TH.decode_term(t, L, N) == ("V", mu, s, nu, sp)
        assert f == 1.0 and blk == sp * N + nu


def test_merged_list_matches_the_oracle(decoded):
    _, terms = decoded
    L = 3
    for (N, merge, t), (mu, s, nu, sp, f, blk) in terms.items():
        if not merge:
            continue
        assert TH.decode_term_merged(t, L, N) == ("V", mu, s, nu, sp, f)
        assert blk == sp * N + nu


def test_reuse_blocks_are_contiguous_and_ascending(decoded):
    # apply_H keeps the reused states of a term range as the slots between the
    # first and the last term's block: the blocks must not decrease along t
    _, terms = decoded
    for N in (1, 2, 3, 5):
        for merge in (0, 1):
            blocks = [terms[(N, merge, t)][5] for t in range(TH.n_coulomb(N, bool(merge)))]
            assert all(b1 >= b0 for b0, b1 in zip(blocks, blocks[1:]))
            assert sorted(set(blocks)) == list(range(2 * N))
