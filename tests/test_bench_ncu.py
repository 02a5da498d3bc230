"""bench.py's readers of ncu CSV logs (host logic, no GPU): DRAM bytes per launch into the
traffic file, and the per-kernel launch table."""
import json

import bench

HDR = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
       '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"')


def _row(i, kernel, metric, unit, value):
    return (f'"{i}","1","python3","h","{kernel}","1","13","(512, 1, 1)","(1024, 1, 1)","0","10.3",'
            f'"Command line profiler metrics","{metric}","{unit}","{value}"')


def _log(tmp_path, name, rows):
    p = tmp_path / name
    p.write_text("==PROF== Connected to process 1\n" + HDR + "\n" + "\n".join(rows) + "\n")
    return str(p)


def test_traffic_labels_launches_in_frame_order(tmp_path):
    k = "k_sort_pass(KParams, DevBufs, const unsigned int *, int)"
    a = _log(tmp_path, "traffic_k_sort_pass.csv", [
        _row(0, k, "dram__bytes_read.sum", "Mbyte", "21.0"), _row(0, k, "dram__bytes_write.sum", "Kbyte", "43"),
        _row(1, k, "dram__bytes_read.sum", "byte", "37,818,112"), _row(1, k, "dram__bytes_write.sum", "byte", "0")])
    s = "void k_segsum_lidar(KParams, DevBufs)"
    b = _log(tmp_path, "traffic_k_segsum_lidar.csv", [
        _row(0, s, "dram__bytes_read.sum", "Mbyte", "102.5"), _row(0, s, "dram__bytes_write.sum", "Mbyte", "63.4")])
    out = tmp_path / "t.json"
    js = bench.write_ncu_traffic([a, b], str(out))
    assert json.loads(out.read_text()) == js
    assert js["csrc_hash"] == bench.csrc_hash()
    rw = js["read_write"]
    assert rw["k_sort_pass0"] == {"read": 21.0e6, "write": 43e3}
    assert rw["k_sort_pass1"] == {"read": 37818112.0, "write": 0.0}
    assert js["kernels"]["k_segsum"] == 102.5e6 + 63.4e6


def test_traffic_rejects_a_capture_of_the_wrong_launch_count(tmp_path):
    k = "k_sort_pass(KParams, DevBufs)"
    a = _log(tmp_path, "x.csv", [_row(0, k, "dram__bytes_read.sum", "byte", "1"),
                                 _row(0, k, "dram__bytes_write.sum", "byte", "1")])
    try:
        bench.write_ncu_traffic([a], str(tmp_path / "t.json"))
    except SystemExit as e:
        assert "k_sort_pass" in str(e)
    else:
        raise AssertionError("one launch of a two-pass sort accepted")


def test_launch_table_sums_per_kernel(tmp_path):
    rows = [_row(i, kn, "gpu__time_duration.sum", "ns", t) for i, (kn, t) in enumerate(
        [("void k_cell<0>(KParams, DevBufs)", "30,000"), ("k_predict(KParams, DevBufs)", "60,000"),
         ("void k_cell<0>(KParams, DevBufs)", "10,000")])]
    table = bench.ncu_launch_table(_log(tmp_path, "l.csv", rows))
    lines = table.splitlines()
    assert lines[2].startswith("| k_predict | 1 | 60.0 | 60.0 | 60.0 % |")
    assert lines[3].startswith("| k_cell | 2 | 40.0 | 20.0 | 40.0 % |")
    assert lines[-1].startswith("| **all** | 3 | 100.0 |")
