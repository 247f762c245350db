"""Seeded synthetic video for tests and benchmarks (no arithmetic of the method)."""
from .video import (VideoSpec, Scene, make_scene, render_frame, generate, pitch_for,
                    SMALL_192x432x60, PARTITIONS_192x432x600, HSDV_800x600x1000)
