"""Seeded synthetic inputs (operators, scenes, noise) shared by the oracle-side
tests and the CUDA-side tests and bench.  No solver arithmetic lives here."""
from .rng import Stream
from .radar import (Geometry, Scene, operator, delays, pixel_centres, sensor_positions,
                    point_targets, cluster_targets, measure, add_noise, lambda_max)
from .configs import (GEOMS, Params, build_scene, scene_law, operators, resolve_lambda, random_problem, batch_geometries,
                      batch_scenes)
from .cnn_init import cnn_init

__all__ = ["Stream", "Geometry", "Scene", "operator", "delays", "pixel_centres",
           "sensor_positions", "point_targets", "cluster_targets", "measure", "add_noise", "lambda_max",
           "GEOMS", "Params", "build_scene", "scene_law", "operators", "resolve_lambda", "random_problem", "batch_geometries",
           "batch_scenes", "cnn_init"]
