"""Host-side summaries of the profiling entry point (no GPU)."""
import json

from paper_1806_00205_gb300 import profile_step as P

HEAD = '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size",' \
       '"Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n'


def row(i, kernel, metric, unit, value):
    return f'"{i}","1","python3","h","{kernel}","1","13","(128, 1, 1)","(1216, 1, 1)","0","10.3",' \
           f'"Command line profiler metrics","{metric}","{unit}","{value}"\n'


TRAV = "void unnamed>::k_traverse_ww<3, 1, 0, 0, 16>(const void *, const float4 *, int)"
SHADE = "void unnamed>::k_shade<0, 1>(const float4 *, TableDesc)"


def test_kernel_label_strips_parameters_and_namespace():
    assert P.kernel_label(TRAV) == "k_traverse_ww<3, 1, 0, 0, 16>"
    assert P.kernel_label("unnamed>::k_morton(const float *, int)") == "k_morton"


def test_launch_summary_shares(tmp_path, capsys):
    f = tmp_path / "l.csv"
    f.write_text("==PROF== Connected\n" + HEAD + row(0, TRAV, "gpu__time_duration.sum", "ns", "3000") +
                 row(1, SHADE, "gpu__time_duration.sum", "ns", "1000") +
                 row(2, TRAV, "gpu__time_duration.sum", "us", "4"))
    P.summarize_launches(str(f))
    out = capsys.readouterr().out.splitlines()
    assert out[2] == "| `k_traverse_ww<3, 1, 0, 0, 16>` | 2 | 0.007 | 87.5 % |"
    assert out[3] == "| `k_shade<0, 1>` | 1 | 0.001 | 12.5 % |"
    assert out[4] == "| all | 3 | 0.008 | 100 % |"


def test_traffic_record_per_hierarchy_ray(tmp_path, capsys):
    f = tmp_path / "d.csv"
    f.write_text(HEAD + row(0, TRAV, "dram__bytes_read.sum", "Mbyte", "1.5") +
                 row(0, TRAV, "dram__bytes_write.sum", "byte", "500000") +
                 row(0, TRAV, "gpu__time_duration.sum", "us", "2") +
                 row(1, SHADE, "dram__bytes_read.sum", "Mbyte", "9") +
                 row(2, TRAV, "dram__bytes_read.sum", "Kbyte", "1000") +
                 row(2, TRAV, "dram__bytes_write.sum", "byte", "0"))
    step = tmp_path / "s.json"
    step.write_text("warming up\n" + json.dumps(dict(
        grid=8, porosity=0.7, n_tri=100, energies=[500.0], angles=[0.0], primaries=10, max_generation=2,
        kernel_sha="abc",
        steps=[dict(hierarchy_rays=30000, rays=40000)])) + "\n")
    P.summarize_traffic(str(f), str(step), 3)
    rec = json.loads(capsys.readouterr().out)
    assert rec["kernel_sha"] == "abc" and rec["node_format"] == 3
    assert len(rec["launches"]) == 2                       # the shade launch is not counted
    assert abs(rec["dram_bytes_per_ray"] - 3.0e6 / 30000) < 1e-9
    assert abs(rec["launches"][0]["ms"] - 0.002) < 1e-12
