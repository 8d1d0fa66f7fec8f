"""The Python binding's ctypes structures and constants against the C header
(no GPU): a small C program built with the system compiler against
include/fsort.h prints every structure's size and field offsets, the status
codes, flags, sizes and kernel kinds; each must equal what the binding uses.
A field added to, moved in or resized in the header without the binding
following would otherwise corrupt every call that passes that structure."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

import paper_2605_10390_gb300 as fs
from paper_2605_10390_gb300 import _binding as b

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))
HEADER = os.path.join(ROOT, "include", "fsort.h")

# C structure name -> ctypes class of the binding
STRUCTS = {
    "fsort_plan_desc": b.FsortPlanDesc,
    "fsort_plan_info": b.FsortPlanInfo,
    "fsort_segment": b.FsortSegment,
    "fsort_batch_config": b.FsortBatchConfig,
    "fsort_learned_opts": b.FsortLearnedOpts,
    "fsort_learned_stats": b.FsortLearnedStats,
    "fsort_serve_desc": b.FsortServeDesc,
    "fsort_request": b.FsortRequest,
    "fsort_result": b.FsortResult,
    "fsort_serve_stats": b.FsortServeStats,
    "fsort_kernel_time": b.FsortKernelTime,
}
C_FIELD = {"pass_": "pass"}  # Python names that differ from the C field names


def _defines(prefix):
    text = open(HEADER).read()
    return sorted(set(re.findall(rf"#define ({prefix}\w+) ", text)))


@pytest.fixture(scope="module")
def layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', f'#include "{HEADER}"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append(f'  printf("size {cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            cf = C_FIELD.get(f, f)
            lines.append(f'  printf("off {cname} {f} %zu\\n", offsetof({cname}, {cf}));')
    for name in ["FSORT_OK", "FSORT_ERR_INVALID_ARG", "FSORT_ERR_OOM", "FSORT_ERR_CUDA", "FSORT_ERR_TIMEOUT",
                 "FSORT_ERR_BUSY", "FSORT_NOT_READY", "FSORT_ERR_INTERNAL", "FSORT_ERR_UNSUPPORTED"]:
        lines.append(f'  printf("status {name} %d\\n", (int){name});')
    for name in _defines("FSORT_FLAG_") + _defines("FSORT_KERNEL_") + ["FSORT_MLP_PARAMS", "FSORT_LEARN_CELLS",
                                                                      "FSORT_LEARN_MAX_HEAVY", "FSORT_NOALLOC_MAX_KEYS"]:
        lines.append(f'  printf("const {name} %llu\\n", (unsigned long long)({name}));')
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi_layout")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    res = {"size": {}, "off": {}, "status": {}, "const": {}}
    for line in out.splitlines():
        kind, *rest = line.split()
        if kind == "off":
            res["off"][(rest[0], rest[1])] = int(rest[2])
        else:
            res[kind][rest[0]] = int(rest[1])
    return res


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_struct_size_and_offsets_match_the_header(layout, cname):
    cls = STRUCTS[cname]
    assert ctypes.sizeof(cls) == layout["size"][cname], cname
    for f, _ in cls._fields_:
        assert getattr(cls, f).offset == layout["off"][(cname, f)], (cname, f)


def test_status_codes_match(layout):
    assert {v: k for k, v in b.STATUS.items()} == layout["status"]


def test_flags_sizes_and_kernel_kinds_match(layout):
    c = layout["const"]
    for name in _defines("FSORT_FLAG_"):
        assert getattr(fs, name) == c[name], name
    assert fs.FSORT_MLP_PARAMS == c["FSORT_MLP_PARAMS"]
    assert fs.FSORT_LEARN_CELLS == c["FSORT_LEARN_CELLS"]
    assert fs.FSORT_LEARN_MAX_HEAVY == c["FSORT_LEARN_MAX_HEAVY"]
    assert fs.FSORT_NOALLOC_MAX_KEYS == c["FSORT_NOALLOC_MAX_KEYS"]
    kinds = {v: k[len("FSORT_KERNEL_"):].lower() for k, v in c.items() if k.startswith("FSORT_KERNEL_")}
    assert kinds == b.KERNEL_KINDS
