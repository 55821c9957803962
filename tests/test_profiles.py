"""The committed ncu summaries: short text files, each giving the full command that made it
(with --clock-control none), and the kernel summaries recording the digest of the kernel
code they were taken on (bench.py reports their DRAM traffic only while it matches)."""
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KERNEL_SUMMARIES = ("translate_tc_fp16x3_shell16.md", "translate_tc_fp16x3_shell32.md",
                    "translate_tc_fp16x3_shell32_sym.md", "translate_simt_fp32_shell32.md",
                    "translate_simt_fp32_shell32_sym.md", "cvfcnn_tc_shell16.md")


def test_profiles_are_short_text_with_their_commands():
    d = os.path.join(ROOT, "profiles")
    for name in os.listdir(d):
        assert name.endswith((".md", ".txt")), name
        text = open(os.path.join(d, name)).read()
        assert len(text) < 16_000, name
        assert "ncu " in text and "--clock-control none" in text, name


def test_kernel_summaries_record_code_digest_and_traffic():
    for name in KERNEL_SUMMARIES:
        text = open(os.path.join(ROOT, "profiles", name)).read()
        assert re.search(r"^kernel_code_sha256_16: [0-9a-f]{16}$", text, re.M), name
        assert re.search(r"^traffic_bytes_per_launch: [0-9]+$", text, re.M), name


def test_kernel_summaries_match_the_current_kernel_code():
    """Every kernel summary was taken on the kernel code as committed: bench.py reads its
    traffic (a stale summary would silently report none)."""
    sys.path.insert(0, ROOT)
    import bench
    source = {"translate_tc": "translate_tc.cu", "translate_simt": "translate_simt.cu", "cvfcnn_tc": "cvfcnn_tc.cu"}
    for name in KERNEL_SUMMARIES:
        src = [v for k, v in source.items() if name.startswith(k)]
        assert len(src) == 1, name
        assert bench.profiled_traffic(name, src[0]) is not None, name
